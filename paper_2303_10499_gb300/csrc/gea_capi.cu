// gea_capi.cu -- context, CUDA-graph step driver and the C ABI declared in
// include/gea.h.
//
// A context owns one device allocation that holds two copies of the state
// (the step reads one and writes the other, so a failed step leaves the last
// completed state intact), the per-step scratch, the multigrid hierarchy and
// the device scalars. One time step is one CUDA graph: the iterations of the
// Jacobi and conjugate-gradient solves run as conditional WHILE nodes whose
// bodies end in a one-thread control kernel, so a step needs no host
// round trip. Two graphs (state 0 -> 1 and state 1 -> 0) are built on the
// first step.
#include "gea_internal.cuh"
#include "gea_debug.cuh"
#include "../../include/gea.h"
#include "../../include/gea_net.h"

#include <nvtx3/nvToolsExt.h>
#include <limits.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

using namespace gea;

struct gea_ctx {
    Geom G;
    Phys F;
    gea_constants C;
    int device = 0;
    cudaStream_t stream = nullptr;        // user stream (launches)
    cudaStream_t cap = nullptr;           // private stream used for graph capture
    cudaStream_t cap2 = nullptr;          // private stream used for loop bodies
    char *mem = nullptr;
    size_t mem_bytes = 0;
    State S[2];
    Stencil9 T;
    double *rho1, *dinvu, *dinvh, *bu, *bw, *ua, *wa, *ub, *wb, *bh, *ha, *hb, *rho2, *psi, *Dx,
        *Dz, *Hx, *Hz, *b, *p0, *p1, *q, *dtr1;
    double *gzc, *gzf;                     // g z of cell-centre rows (nz) and z-face rows (nz + 1)
    double *stage;                         // staging for conservative set/get (4 fields)
    size_t stage_stride = 0;               // elements from one staging field to the next
    double *thbar;                         // nz values
    double *thout;                         // theta' output
    std::vector<Level> L;                 // FP64 hierarchy (mixed precision: the finest level only)
    bool mixed = false;                   // GEA_FLAG_MIXED
    MixedArgs mx{};                       // FP32 buffers of the mixed-precision step
    std::vector<LevelF> Lf;               // FP32 hierarchy of the mixed-precision step
    double *r0keep = nullptr;             // GEA_FLAG_KEEP_R0: first corrector's initial residual
    double *mueff = nullptr;              // LES: mu + mu_t of the running step
    gea_net *net = nullptr;               // attached learned network (not owned)
    int net_mode = 0;                     // 1: initial guess; 2: flexible-CG preconditioner; 3: both
    double *net_s = nullptr;              // mode 2: the residual the network leaves (V-cycle input)
    int tiles_per_block = 0;              // per-phase reduction kernels (0: the size rule)
    float *net_r = nullptr, *net_e = nullptr;   // its dense input and output
    Scal *sc = nullptr;
    double *partials = nullptr;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t ev[8];
    int nev = 0;
    bool have_state = false;
    int base = 0;                         // state slot loaded by the last set_state
    int pers_blocks = 0;                  // persistent-kernel grid (0: graph path only)
    long long wait_polls = -1;            // grid-barrier poll limit of the persistent kernels (< 0: default)
    unsigned long long *trace = nullptr;  // phase trace of the persistent kernels (gea_set_trace; not owned)
    int trace_bars = 0;
    int shape = SHAPE_32x8;               // tile shape of the persistent kernels (gea_set_tile_shape)
    long long steps_at_sync = 0;          // device steps_done at the last sync
    // GEA_FLAG_DEBUG_PADS: the pitched arrays, on the host and the device,
    // and the check results (two: per-launch tracking, final count)
    std::vector<gea_pad_region> pads;
    PadRegionDev *dpads = nullptr;
    PadResult *dpres = nullptr;
    char err[256] = {0};
};

namespace {

int fail(gea_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, GEA_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                               \
    } while (0)

size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

Geom make_geom(int nx, int nz, double lx, double lz)
{
    Geom G;
    G.nx = nx;
    G.nz = nz;
    G.P = (int)round_up((size_t)nx + 1, 32);
    G.dx = lx / nx;
    G.dz = lz / nz;
    G.idx = 1.0 / G.dx;
    G.idz = 1.0 / G.dz;
    G.iV = 1.0 / (G.dx * G.dz);
    return G;
}

// bytes of one pitched array with `rows` rows
size_t arr_bytes(const Geom &G, int rows) { return round_up((size_t)G.P * rows * sizeof(double), 256); }
size_t arr_bytes_f(const Geom &G, int rows) { return round_up((size_t)G.P * rows * sizeof(float), 256); }

StepArgs step_args(gea_ctx *c, int from)
{
    StepArgs a;
    a.G = c->G;
    a.F = c->F;
    a.S = c->S[from];
    a.N = c->S[from ^ 1];
    a.T = c->T;
    a.mueff = c->mueff;
    a.rho1 = c->rho1; a.dinvu = c->dinvu; a.dinvh = c->dinvh; a.bu = c->bu; a.bw = c->bw;
    a.ua = c->ua; a.wa = c->wa; a.ub = c->ub; a.wb = c->wb;
    a.bh = c->bh; a.ha = c->ha; a.hb = c->hb;
    a.rho2 = c->rho2; a.psi = c->psi; a.Dx = c->Dx; a.Dz = c->Dz; a.Hx = c->Hx; a.Hz = c->Hz;
    a.b = c->b; a.p0 = c->p0; a.p1 = c->p1; a.q = c->q;
    a.dtr1 = c->dtr1;
    a.gzc = c->gzc;
    a.gzf = c->gzf;
    a.sc = c->sc;
    a.partials = c->partials;
    a.jac_rtol2 = c->C.jac_rtol * c->C.jac_rtol;
    a.cg_rtol2 = c->C.cg_rtol * c->C.cg_rtol;
    a.tiles_per_block = c->tiles_per_block;
    a.trace = c->trace;
    a.trace_bars = c->trace_bars;
    return a;
}

constexpr int kCoarseSweeps = 2;   // damped Jacobi sweeps on the coarsest level (even)
constexpr double kOmega = 0.8;     // smoother weight
// The multigrid hierarchy stops once the Laplacian part of the Helmholtz
// operator is small against its diagonal psi/dt: with D ~ dt and psi ~ 1/(RT),
// sum_f a_f / c ~ 2 dt^2 R T (1/dx^2 + 1/dz^2), and every coarsening divides
// it by 4. Coarsening continues while the ratio exceeds this bound.
constexpr double kCoarsestRatio = 1.0;
constexpr double kRefT = 300.0;    // reference temperature of that estimate (K)
constexpr int kPersistTilesPerBlock = 4;
constexpr double kMixedRtol = 1e-5;  // default tolerance of the FP32 solves (relative to ||r0||)

// Append a WHILE conditional node to the graph being captured on `s`; its
// body is captured from body(body_stream, handle, true).
template <class Body>
int capture_while(gea_ctx *ctx, cudaStream_t s, Body body, int gate = -1)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) return fail(ctx, GEA_ERR_CUDA, "capture not active");
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    if (gate >= 0) {
        // a gated loop runs no trip when it is already finished: a kernel
        // ahead of the node sets the condition from the loop's flags
        launch_loop_gate(ctx->sc, h, gate, s);
        CK(cudaGetLastError());
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &ndeps));
    }
    cudaGraphNodeParams prm = {cudaGraphNodeTypeConditional};
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, edges, ndeps, &prm));
    cudaGraph_t bodyg = prm.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK(cudaStreamBeginCaptureToGraph(ctx->cap2, bodyg, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    body(ctx->cap2, h, true);
    cudaGraph_t out = nullptr;
    CK(cudaStreamEndCapture(ctx->cap2, &out));
    return GEA_OK;
}

// The learned initial guess of a pressure solve: convert r0 for the network
// and, in a graph, run the network and the step under an IF node that the
// conversion kernel sets (skipped when the solve has already converged);
// eagerly, skip them on the host in that case. Returns kernels launched
// outside loops, or a negative value on failure.
template <class R>
int record_guess(gea_ctx *ctx, const StepArgs &a, const LevelT<R> &L, R *q, R *x, double tol2, cudaStream_t s,
                 bool graph, Tracer *tr)
{
    if (!graph) {
        launch_guess_in<R>(a, L, L.r, ctx->net_r, (cudaGraphConditionalHandle)0, false, s, tr);
        Scal h;
        if (cudaMemcpyAsync(&h, ctx->sc, sizeof(Scal), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return -1;
        if (h.done[LOOP_CG] || h.status) return 1;
        const int k = launch_net_guess<R>(a, L, L.r, q, x, tol2, ctx->net, ctx->net_r, ctx->net_e, s, tr);
        return k < 0 ? -1 : 1 + k;
    }
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &ndeps) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
        return -1;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) return -1;
    launch_guess_in<R>(a, L, L.r, ctx->net_r, h, true, s, tr);
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &ndeps) != cudaSuccess) return -1;
    cudaGraphNodeParams prm = {cudaGraphNodeTypeConditional};
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeIf;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps, edges, ndeps, &prm) != cudaSuccess) return -1;
    cudaGraph_t bodyg = prm.conditional.phGraph_out[0];
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
            cudaSuccess ||
        cudaStreamBeginCaptureToGraph(ctx->cap2, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess)
        return -1;
    const int k = launch_net_guess<R>(a, L, L.r, q, x, tol2, ctx->net, ctx->net_r, ctx->net_e, ctx->cap2, tr);
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(ctx->cap2, &out) != cudaSuccess || k < 0) return -1;
    // the launches of the IF body are not counted (they may not run)
    return 1;
}

// Run a loop body eagerly on `s` until its control kernel reports that the
// loop is finished (converged, failed or at its trip cap).
template <class Body>
int eager_while(gea_ctx *ctx, cudaStream_t s, int which, int maxtrips, Body body, bool gated = false)
{
    if (gated) {
        Scal h;
        CK(cudaMemcpyAsync(&h, ctx->sc, sizeof(Scal), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h.done[which] || h.status) return GEA_OK;
    }
    for (int t = 0; t < maxtrips + 1; ++t) {
        body(s, (cudaGraphConditionalHandle)0, false);
        Scal h;
        CK(cudaMemcpyAsync(&h, ctx->sc, sizeof(Scal), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h.done[which] || h.status || h.trips[which] >= maxtrips) break;
    }
    return GEA_OK;
}

// The kernel sequence of one time step reading state `from` and writing
// state `from ^ 1` (Section 3: Step 1, Step 2, then n_corr PISO correctors).
// graph = true: enqueue into the capture running on s (loops become WHILE
// nodes); graph = false: launch eagerly with host-checked loops, every launch
// bracketed by tr.
int record_step(gea_ctx *ctx, int from, cudaStream_t s, bool graph, Tracer *tr)
{
    StepArgs a = step_args(ctx, from);
    Level *L = ctx->L.data();
    const int nlev = (int)ctx->L.size();
    const int jtrips = (ctx->C.jac_maxit + 1) / 2;
    int fixed = 0;
    int rc = GEA_OK;
    auto loop = [&](int which, int maxtrips, auto body) {
        return graph ? capture_while(ctx, s, body) : eager_while(ctx, s, which, maxtrips, body);
    };

    launch_step_begin(ctx->sc, s, tr); ++fixed;
    if (ctx->mueff) { launch_les(a, s, tr); ++fixed; }
    // Step 1: continuity predictor and implicit momentum predictor
    launch_pred_setup(a, s, tr); ++fixed;
    rc = loop(LOOP_MOM, jtrips, [&](cudaStream_t bs, cudaGraphConditionalHandle h, bool g) {
        launch_mom_jacobi(a, a.ua, a.wa, a.ub, a.wb, 0, bs, tr);
        launch_mom_jacobi(a, a.ub, a.wb, a.ua, a.wa, 1, bs, tr);
        launch_loop_ctl(a.sc, h, g, LOOP_MOM, jtrips, 3, bs, tr);
    });
    if (rc) return rc;
    // Step 2: enthalpy, temperature, rho^{n+2/3}
    launch_enth_rhs(a, s, tr); ++fixed;
    rc = loop(LOOP_ENTH, jtrips, [&](cudaStream_t bs, cudaGraphConditionalHandle h, bool g) {
        launch_enth_jacobi(a, a.ha, a.hb, 0, bs, tr);
        launch_enth_jacobi(a, a.hb, a.ha, 1, bs, tr);
        launch_loop_ctl(a.sc, h, g, LOOP_ENTH, jtrips, 3, bs, tr);
    });
    if (rc) return rc;
    launch_eos_coef(a, L[0], s, tr); ++fixed;
    for (int l = 0; l + 1 < nlev; ++l) { launch_mg_coarsen(L[l], L[l + 1], ctx->F.omega, s, tr); ++fixed; }
    // Step 3: PISO correctors
    const int body_cg = (nlev == 1 ? 2 : 2 + (nlev - 2) + kCoarseSweeps + (nlev - 1)) + 1;
    for (int c = 0; c < ctx->C.n_corr; ++c) {
        const double *U = c == 0 ? a.ua : a.N.u;
        const double *W = c == 0 ? a.wa : a.N.w;
        launch_H(a, U, W, s, tr); ++fixed;
        // inside a capture an event record becomes a timing node only when
        // recorded as external
        CK(graph ? cudaEventRecordWithFlags(ctx->ev[2 * c], s, cudaEventRecordExternal)
                 : cudaEventRecord(ctx->ev[2 * c], s));
        launch_helm_rhs(a, L[0], c == 0 ? a.S.pp : a.N.pp, a.N.pp, c, s, tr); ++fixed;
        if (ctx->r0keep && c == 0)
            CK(cudaMemcpyAsync(ctx->r0keep, L[0].r, arr_bytes(ctx->G, ctx->G.nz), cudaMemcpyDeviceToDevice, s));
        if (ctx->net && (ctx->net_mode & 1)) {
            const int k = record_guess<double>(ctx, a, L[0], a.q, a.N.pp, a.cg_rtol2, s, graph, tr);
            if (k < 0) return fail(ctx, GEA_ERR_CUDA, "learned initial guess failed");
            fixed += k;
        }
        if (ctx->net && (ctx->net_mode & 2)) {
            // flexible CG with the two-stage preconditioner (the network,
            // then a V-cycle on what it leaves): each trip preconditions the
            // current residual, then steps; gated, so that a solve that is
            // already converged runs no network pass
            int bad = 0;
            auto body = [&](cudaStream_t bs, cudaGraphConditionalHandle h, bool g) {
                const int nb = launch_fcg_iter(a, L, nlev, kCoarseSweeps, a.N.pp, ctx->net, ctx->net_r,
                                               ctx->net_e, ctx->net_s, bs, tr);
                if (nb < 0) bad = 1;
                launch_loop_ctl(a.sc, h, g, LOOP_CG, ctx->C.cg_maxit, nb < 0 ? 0 : nb + 1, bs, tr);
            };
            rc = graph ? capture_while(ctx, s, body, LOOP_CG)
                       : eager_while(ctx, s, LOOP_CG, ctx->C.cg_maxit, body, true);
            if (graph) ++fixed;   // the gate kernel
            if (rc) return rc;
            if (bad) return fail(ctx, GEA_ERR_CUDA, "network preconditioner failed");
        } else {
            fixed += launch_vcycle(a, L, nlev, kCoarseSweeps, s, tr);   // z = M^-1 r_0
            rc = loop(LOOP_CG, ctx->C.cg_maxit, [&](cudaStream_t bs, cudaGraphConditionalHandle h, bool g) {
                launch_cg_iter(a, L, nlev, kCoarseSweeps, a.N.pp, bs, tr);
                launch_loop_ctl(a.sc, h, g, LOOP_CG, ctx->C.cg_maxit, body_cg, bs, tr);
            });
            if (rc) return rc;
        }
        CK(graph ? cudaEventRecordWithFlags(ctx->ev[2 * c + 1], s, cudaEventRecordExternal)
                 : cudaEventRecord(ctx->ev[2 * c + 1], s));
        launch_correct(a, s, tr); ++fixed;
    }
    ++fixed;
    launch_step_end(ctx->sc, fixed, s, tr);
    return GEA_OK;
}

// The mixed-precision step: the same phases, with the three linear solves
// done as FP64 residual + FP32 solve for the increment + FP64 update. The
// increments du, dw (Step 1) and dh (Step 2) run their Jacobi sweeps in
// pairs that end in du[0], dw[0], dh[0]; the pressure increment accumulates
// in mx.x and is added to p' before the correction.
int record_step_mixed(gea_ctx *ctx, int from, cudaStream_t s, bool graph, Tracer *tr)
{
    StepArgs a = step_args(ctx, from);
    const MixedArgs &m = ctx->mx;
    Level &L0 = ctx->L[0];
    LevelF *Lf = ctx->Lf.data();
    const int nlev = (int)ctx->Lf.size();
    const int jtrips = (ctx->C.jac_maxit + 1) / 2;
    int fixed = 0;
    int rc = GEA_OK;
    auto loop = [&](int which, int maxtrips, auto body) {
        return graph ? capture_while(ctx, s, body) : eager_while(ctx, s, which, maxtrips, body);
    };

    launch_step_begin(ctx->sc, s, tr); ++fixed;
    if (ctx->mueff) { launch_les(a, s, tr); ++fixed; }
    launch_mx_pred(a, m, s, tr); ++fixed;
    rc = loop(LOOP_MOM, jtrips, [&](cudaStream_t bs, cudaGraphConditionalHandle h, bool g) {
        launch_mx_mom(a, m, m.du[0], m.dw[0], m.du[1], m.dw[1], 0, bs, tr);
        launch_mx_mom(a, m, m.du[1], m.dw[1], m.du[0], m.dw[0], 1, bs, tr);
        launch_loop_ctl(a.sc, h, g, LOOP_MOM, jtrips, 3, bs, tr);
    });
    if (rc) return rc;
    launch_mx_enth_rhs(a, m, s, tr); ++fixed;
    rc = loop(LOOP_ENTH, jtrips, [&](cudaStream_t bs, cudaGraphConditionalHandle h, bool g) {
        launch_mx_enth(a, m, m.dh[0], m.dh[1], 0, bs, tr);
        launch_mx_enth(a, m, m.dh[1], m.dh[0], 1, bs, tr);
        launch_loop_ctl(a.sc, h, g, LOOP_ENTH, jtrips, 3, bs, tr);
    });
    if (rc) return rc;
    launch_mx_eos(a, L0, Lf[0], m.dh[0], s, tr); ++fixed;
    for (int l = 0; l + 1 < nlev; ++l) { launch_mx_coarsen(Lf[l], Lf[l + 1], ctx->F.omega, s, tr); ++fixed; }
    const int body_cg = (nlev == 1 ? 2 : 2 + (nlev - 2) + kCoarseSweeps + (nlev - 1)) + 1;
    for (int c = 0; c < ctx->C.n_corr; ++c) {
        const double *U = c == 0 ? a.ua : a.N.u;
        const double *W = c == 0 ? a.wa : a.N.w;
        launch_H(a, U, W, s, tr); ++fixed;
        CK(graph ? cudaEventRecordWithFlags(ctx->ev[2 * c], s, cudaEventRecordExternal)
                 : cudaEventRecord(ctx->ev[2 * c], s));
        launch_mx_helm_rhs(a, L0, Lf[0], m, c == 0 ? a.S.pp : a.N.pp, a.N.pp, c, s, tr); ++fixed;
        if (ctx->net && (ctx->net_mode & 1)) {
            const int k = record_guess<float>(ctx, a, Lf[0], m.q, m.x, m.tol2, s, graph, tr);
            if (k < 0) return fail(ctx, GEA_ERR_CUDA, "learned initial guess failed");
            fixed += k;
        }
        fixed += launch_mx_vcycle(a, Lf, nlev, kCoarseSweeps, s, tr);
        rc = loop(LOOP_CG, ctx->C.cg_maxit, [&](cudaStream_t bs, cudaGraphConditionalHandle h, bool g) {
            launch_mx_cg_iter(a, m, Lf, nlev, kCoarseSweeps, bs, tr);
            launch_loop_ctl(a.sc, h, g, LOOP_CG, ctx->C.cg_maxit, body_cg, bs, tr);
        });
        if (rc) return rc;
        launch_mx_p_apply(a, m, s, tr); ++fixed;
        CK(graph ? cudaEventRecordWithFlags(ctx->ev[2 * c + 1], s, cudaEventRecordExternal)
                 : cudaEventRecord(ctx->ev[2 * c + 1], s));
        launch_correct(a, s, tr); ++fixed;
    }
    ++fixed;
    launch_step_end(ctx->sc, fixed, s, tr);
    return GEA_OK;
}

int record_any(gea_ctx *ctx, int from, cudaStream_t s, bool graph, Tracer *tr)
{
    return ctx->mixed ? record_step_mixed(ctx, from, s, graph, tr) : record_step(ctx, from, s, graph, tr);
}

int build_graph(gea_ctx *ctx, int from)
{
    cudaStream_t s = ctx->cap;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = record_any(ctx, from, s, true, nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(ctx, GEA_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    ctx->graph[from] = g;
    CK(cudaGraphInstantiate(&ctx->exec[from], g, 0));
    return GEA_OK;
}

int ensure_graphs(gea_ctx *ctx)
{
    for (int f = 0; f < 2; ++f)
        if (!ctx->exec[f]) {
            int rc = build_graph(ctx, f);
            if (rc) return rc;
        }
    return GEA_OK;
}

// Records an event pair around every launch of an eager step, inside an
// NVTX range named after the kernel (visible to a timeline profiler). A
// kernel of a solver loop returns at once when its loop has already
// finished (the solve converged inside the loop body, or the second Jacobi
// sweep of a pair copies after the first met the tolerance): such a launch is
// recorded with zero cells, so that the per-cell work models count only
// launches that did the work (the loop's flags are read before the launch;
// the profiled step synchronises anyway).
struct EventTracer : Tracer {
    struct Rec {
        const char *name;
        long long cells;
        cudaEvent_t e0, e1;
    };
    std::vector<Rec> recs;
    const Scal *dsc;
    explicit EventTracer(const Scal *sc) : dsc(sc) {}
    // the loop whose finished flag makes the kernel return, or -1
    static int gate(const char *name)
    {
        static const char *cg[] = {"mg_down", "mg_coarse", "mg_up", "mg_single", "cg_pspmv", "cg_update_single",
                                   "cg_update_down", "mx_mg_down", "mx_mg_coarse", "mx_mg_up", "mx_mg_single",
                                   "mx_pspmv", "mx_update_single", "mx_update_down"};
        for (const char *c : cg)
            if (!strcmp(name, c)) return LOOP_CG;
        if (!strcmp(name, "mom_jacobi") || !strcmp(name, "mx_mom")) return LOOP_MOM;
        if (!strcmp(name, "enth_jacobi") || !strcmp(name, "mx_enth")) return LOOP_ENTH;
        return -1;
    }
    void begin(const char *name, long long cells, cudaStream_t st) override
    {
        const int g = gate(name);
        if (g >= 0) {
            Scal h;
            if (cudaMemcpyAsync(&h, dsc, sizeof(Scal), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                cudaStreamSynchronize(st) == cudaSuccess && (h.status || h.done[g]))
                cells = 0;
        }
        Rec r{name, cells, nullptr, nullptr};
        nvtxRangePushA(name);
        cudaEventCreate(&r.e0);
        cudaEventCreate(&r.e1);
        cudaEventRecord(r.e0, st);
        recs.push_back(r);
    }
    void end(cudaStream_t st) override
    {
        cudaEventRecord(recs.back().e1, st);
        nvtxRangePop();
    }
    ~EventTracer() override
    {
        for (auto &r : recs) {
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
    }
};

// Checks every pad of a GEA_FLAG_DEBUG_PADS context after every launch of
// an eager step (check ordinal = the launch's index).
struct PadTracer : Tracer {
    gea_ctx *ctx;
    std::vector<const char *> names;
    cudaError_t err = cudaSuccess;
    explicit PadTracer(gea_ctx *c) : ctx(c) {}
    void begin(const char *name, long long, cudaStream_t) override { names.push_back(name); }
    void end(cudaStream_t st) override
    {
        cudaError_t e = launch_pad_check(ctx->dpads, (int)ctx->pads.size(), ctx->dpres, (int)names.size() - 1, st);
        if (err == cudaSuccess) err = e;
    }
};

int read_scal(gea_ctx *ctx, Scal *h)
{
    CK(cudaMemcpyAsync(h, ctx->sc, sizeof(Scal), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GEA_OK;
}

int current_slot(gea_ctx *ctx, const Scal &h)
{
    return (int)((ctx->base + h.steps_done) & 1);
}

// Pitched copy of a dense nz x ncols host/device array to/from device.
int copy_in(gea_ctx *ctx, double *dst, const double *src, int ncols, int rows)
{
    CK(cudaMemcpy2DAsync(dst, (size_t)ctx->G.P * sizeof(double), src, (size_t)ncols * sizeof(double),
                         (size_t)ncols * sizeof(double), rows, cudaMemcpyDefault, ctx->stream));
    return GEA_OK;
}
int copy_out(gea_ctx *ctx, double *dst, const double *src, int ncols, int rows)
{
    CK(cudaMemcpy2DAsync(dst, (size_t)ncols * sizeof(double), src, (size_t)ctx->G.P * sizeof(double),
                         (size_t)ncols * sizeof(double), rows, cudaMemcpyDefault, ctx->stream));
    return GEA_OK;
}

}  // namespace

extern "C" {

int gea_create(const gea_grid *grid, const gea_constants *c, gea_ctx **out)
{
    gea_ctx *ctx = nullptr;
    if (!grid || !c || !out) return GEA_ERR_INVAL;
    *out = nullptr;
    if (grid->nx < 4 || grid->nz < 4 || !(grid->lx > 0) || !(grid->lz > 0)) return GEA_ERR_INVAL;
    if ((long long)grid->nx * grid->nz > (1LL << 31) / 2) return GEA_ERR_INVAL;
    // the grid sums' group counters cover this many tiles (blocks)
    if ((long long)((grid->nx + BX - 1) / BX) * ((grid->nz + BZ - 1) / BZ) > (long long)kGroupCounters * kSumGroup)
        return GEA_ERR_INVAL;
    if (!(c->R > 0) || !(c->cp > c->R) || !(c->g >= 0) || !(c->p0 > 0) || !(c->mu >= 0) ||
        !(c->Pr > 0) || !(c->dt > 0) || c->n_corr < 1 || c->n_corr > 4 || !(c->jac_rtol > 0) ||
        c->jac_maxit < 1 || !(c->cg_rtol > 0) || c->cg_maxit < 1 || c->mg_min_cells < 0 ||
        (c->flags & ~(GEA_FLAG_GRAPH | GEA_FLAG_MIXED | GEA_FLAG_KEEP_R0 | GEA_FLAG_DEBUG_PADS)) ||
        (c->reading_flags & ~(uint32_t)GEA_READING_K_LAGGED) ||
        ((c->flags & GEA_FLAG_KEEP_R0) && (c->flags & GEA_FLAG_MIXED)))
        return GEA_ERR_INVAL;
    if ((c->flags & GEA_FLAG_MIXED) && c->mp_rtol != 0.0 && !(c->mp_rtol >= 1e-7 && c->mp_rtol < 1.0))
        return GEA_ERR_INVAL;
    // LES: one viscosity field serves momentum and enthalpy, so Pr = 1
    if (!(c->cs >= 0.0) || (c->cs > 0.0 && c->Pr != 1.0)) return GEA_ERR_INVAL;

    ctx = new gea_ctx();
    ctx->C = *c;
    ctx->G = make_geom(grid->nx, grid->nz, grid->lx, grid->lz);
    ctx->F.les_d2 = c->cs * c->cs * ctx->G.dx * ctx->G.dz;
    ctx->F.R = c->R; ctx->F.cp = c->cp; ctx->F.g = c->g; ctx->F.p0 = c->p0;
    ctx->F.mu = c->mu; ctx->F.nuh = c->mu / c->Pr; ctx->F.dt = c->dt; ctx->F.idt = 1.0 / c->dt;
    ctx->F.k_lagged = (c->reading_flags & GEA_READING_K_LAGGED) ? 1 : 0;
    ctx->F.les = ctx->F.les_d2 > 0.0 ? 1 : 0;
    ctx->F.pr_ne1 = ctx->F.nuh != ctx->F.mu ? 1 : 0;
    ctx->mixed = (c->flags & GEA_FLAG_MIXED) != 0;
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        delete ctx;
        return GEA_ERR_CUDA;
    }

    // multigrid levels: halve while both sizes are even, the level is larger
    // than mg_min_cells (if given) and the estimated Laplacian-to-diagonal
    // ratio of the Helmholtz operator exceeds kCoarsestRatio
    std::vector<Geom> lg;
    lg.push_back(ctx->G);
    double ratio = 2.0 * c->dt * c->dt * c->R * kRefT * (ctx->G.idx * ctx->G.idx + ctx->G.idz * ctx->G.idz);
    while (true) {
        const Geom &f = lg.back();
        if (f.nx % 2 || f.nz % 2 || f.nx < 8 || f.nz < 8) break;
        if (c->mg_min_cells > 0 && (long long)f.nx * f.nz <= c->mg_min_cells) break;
        if (c->mg_min_cells == 0 && ratio <= kCoarsestRatio) break;
        if ((int)lg.size() >= kMaxLevels) break;
        lg.push_back(make_geom(f.nx / 2, f.nz / 2, f.nx * f.dx, f.nz * f.dz));
        ratio *= 0.25;
    }
    // Jacobi weight: omega damps the smoother of a multigrid hierarchy; a
    // one-level preconditioner is two undamped sweeps (omega = 1), whose
    // preconditioned operator lambda (2 - lambda) on the spectrum of D^-1 A
    // (inside its Gershgorin interval [1 - rho, 1 + rho], rho < 1) is the
    // degree-2 Chebyshev polynomial of that interval up to a factor, which
    // CG does not see: condition number 1 / (1 - rho^2) for any rho, against
    // (1 - (1 - omega (1 + rho))^2) / (1 - (1 - omega (1 - rho))^2) for two
    // damped sweeps (1.28 against 1.50 at rho = 0.47, omega = 0.8)
    ctx->F.omega = lg.size() == 1 ? 1.0 : kOmega;

    // one allocation for everything
    const Geom &G = ctx->G;
    const size_t cell = arr_bytes(G, G.nz), fz = arr_bytes(G, G.nz + 1);
    size_t total = 0;
    total += 2 * (10 * cell + fz);                 // two states (phiz has nz+1 rows)
    total += 34 * cell + 2 * fz;                   // scratch (Dz has nz+1 rows)
    total += round_up((2 * (size_t)G.nz + 1) * sizeof(double), 256);   // height tables
    total += 4 * cell;                             // staging for conservative fields
    total += 2 * cell + round_up(G.nz * sizeof(double), 256);   // theta_bar, theta'
    if (c->flags & GEA_FLAG_KEEP_R0) total += cell;
    if (c->cs > 0.0) total += cell;
    // FP64 levels (mixed precision: the finest only, for the FP64 residual)
    const size_t nlev64 = ctx->mixed ? 1 : lg.size();
    for (size_t l = 0; l < nlev64; ++l) total += 8 * arr_bytes(lg[l], lg[l].nz) + arr_bytes(lg[l], lg[l].nz + 1);
    const size_t cellf = arr_bytes_f(G, G.nz);
    if (ctx->mixed) {
        total += 24 * cellf;                                        // MixedArgs
        for (const Geom &g : lg) total += 8 * arr_bytes_f(g, g.nz) + arr_bytes_f(g, g.nz + 1);
    }
    // reduction partials: the per-phase kernels' grid sums need one slot per
    // 32 x 8 tile, the persistent kernels two buffers of kRedVals per block
    // (at most one block per tile of their shape)
    const size_t nb = (size_t)max_blocks(G);
    size_t nb_all = nb;
    for (int sh = 0; sh < NSHAPES; ++sh) {
        const PersistOps &o = persist_ops(sh);
        nb_all = std::max(nb_all, (size_t)shape_tiles(G, o.bx, o.bz));
    }
    total += round_up((kGcntDoubles + 8 * nb_all) * sizeof(double), 256);   // group counters, reduction partials
    total += round_up(sizeof(Scal), 256);
    const bool dbg = (c->flags & GEA_FLAG_DEBUG_PADS) != 0;
    const size_t guard = dbg ? GEA_PAD_GUARD_BYTES : 0;
    if (dbg) total += guard * (kMaxPadRegions + 1);
    ctx->mem_bytes = total;
    if (cudaMalloc(&ctx->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return GEA_ERR_NOMEM;
    }
    cudaMemset(ctx->mem, 0, total);
    char *ptr = ctx->mem + guard;
    auto take = [&](size_t bytes) { double *r = (double *)ptr; ptr += bytes; return r; };
    // one pitched array (rows x cols in use, the level's pitch), recorded
    // for pad checking, with the guard band behind it
    auto arr = [&](const Geom &g, int rows, int cols, int esize, const char *fmt, int i) -> char * {
        const size_t bytes = round_up((size_t)g.P * rows * esize, 256);
        char *r = ptr;
        ptr += bytes + guard;
        if (dbg && ctx->pads.size() < (size_t)kMaxPadRegions) {
            gea_pad_region pr;
            memset(&pr, 0, sizeof(pr));
            snprintf(pr.name, sizeof(pr.name), fmt, i);
            pr.ptr = r;
            pr.elem_bytes = esize;
            pr.pitch = g.P;
            pr.rows = rows;
            pr.cols = cols;
            pr.span = (int64_t)((bytes + guard) / esize);
            ctx->pads.push_back(pr);
        }
        return r;
    };
    // a vector of n doubles (one row of n)
    auto vec = [&](size_t n, const char *name) -> double * {
        Geom g1 = G;
        g1.P = (int)n;
        return (double *)arr(g1, 1, (int)n, 8, name, 0);
    };
    const int nx = G.nx, nz = G.nz;
    auto cellA = [&](const char *fmt, int i) { return (double *)arr(G, nz, nx, 8, fmt, i); };
    for (int s = 0; s < 2; ++s) {
        State &S = ctx->S[s];
        S.rho = cellA("S%d.rho", s); S.u = cellA("S%d.u", s); S.w = cellA("S%d.w", s);
        S.T = cellA("S%d.T", s); S.h = cellA("S%d.h", s); S.p = cellA("S%d.p", s);
        S.pp = cellA("S%d.pp", s); S.pold = cellA("S%d.pold", s);
        S.phix = (double *)arr(G, nz, nx + 1, 8, "S%d.phix", s);
        S.phiz = (double *)arr(G, nz + 1, nx, 8, "S%d.phiz", s);
        S.Kold = cellA("S%d.Kold", s);
    }
    Stencil9 &T = ctx->T;
    T.cC = cellA("T.cC", 0); T.cE1 = cellA("T.cE1", 0); T.cE2 = cellA("T.cE2", 0); T.cW1 = cellA("T.cW1", 0);
    T.cW2 = cellA("T.cW2", 0); T.cN1 = cellA("T.cN1", 0); T.cN2 = cellA("T.cN2", 0); T.cS1 = cellA("T.cS1", 0);
    T.cS2 = cellA("T.cS2", 0);
    ctx->rho1 = cellA("rho1", 0); ctx->dinvu = cellA("dinvu", 0); ctx->dinvh = cellA("dinvh", 0);
    ctx->bu = cellA("bu", 0); ctx->bw = cellA("bw", 0);
    ctx->ua = cellA("ua", 0); ctx->wa = cellA("wa", 0); ctx->ub = cellA("ub", 0); ctx->wb = cellA("wb", 0);
    ctx->bh = cellA("bh", 0); ctx->ha = cellA("ha", 0); ctx->hb = cellA("hb", 0); ctx->rho2 = cellA("rho2", 0);
    ctx->psi = cellA("psi", 0);
    ctx->Dx = (double *)arr(G, nz, nx + 1, 8, "Dx", 0);
    ctx->Dz = (double *)arr(G, nz + 1, nx, 8, "Dz", 0);
    ctx->Hx = cellA("Hx", 0); ctx->Hz = cellA("Hz", 0); ctx->b = cellA("b", 0);
    ctx->p0 = cellA("p0", 0); ctx->p1 = cellA("p1", 0); ctx->q = cellA("q", 0);
    ctx->dtr1 = cellA("dtr1", 0);
    ctx->gzc = vec(2 * (size_t)nz + 1, "gz");
    ctx->gzf = ctx->gzc + nz;
    ctx->stage = cellA("stage%d", 0);
    for (int j = 1; j < 4; ++j) cellA("stage%d", j);
    ctx->stage_stride = (arr_bytes(G, nz) + guard) / sizeof(double);
    ctx->thout = cellA("thout", 0);
    ctx->thbar = vec(nz, "thbar");
    if (c->flags & GEA_FLAG_KEEP_R0) ctx->r0keep = cellA("r0keep", 0);
    if (c->cs > 0.0) ctx->mueff = cellA("mueff", 0);
    for (size_t lv = 0; lv < nlev64; ++lv) {
        const Geom &g = lg[lv];
        const int l_ = (int)lv;
        Level l;
        l.G = g;
        auto la = [&](const char *fmt) { return (double *)arr(g, g.nz, g.nx, 8, fmt, l_); };
        l.c = la("L%d.c"); l.d = la("L%d.d"); l.wd = la("L%d.wd");
        l.ax = (double *)arr(g, g.nz, g.nx + 1, 8, "L%d.ax", l_);
        l.az = (double *)arr(g, g.nz + 1, g.nx, 8, "L%d.az", l_);
        l.r = la("L%d.r"); l.e = la("L%d.e"); l.e2 = la("L%d.e2"); l.r_alt = la("L%d.r_alt");
        ctx->L.push_back(l);
    }
    if (ctx->mixed) {
        auto cellF = [&](const char *fmt, int i) { return (float *)arr(G, nz, nx, 4, fmt, i); };
        MixedArgs &m = ctx->mx;
        Stencil9F &T32 = m.T;
        T32.cC = cellF("F.T.cC", 0); T32.cE1 = cellF("F.T.cE1", 0); T32.cE2 = cellF("F.T.cE2", 0);
        T32.cW1 = cellF("F.T.cW1", 0); T32.cW2 = cellF("F.T.cW2", 0); T32.cN1 = cellF("F.T.cN1", 0);
        T32.cN2 = cellF("F.T.cN2", 0); T32.cS1 = cellF("F.T.cS1", 0); T32.cS2 = cellF("F.T.cS2", 0);
        m.dinvu = cellF("F.dinvu", 0); m.dinvh = cellF("F.dinvh", 0);
        m.r0u = cellF("F.r0u", 0); m.r0w = cellF("F.r0w", 0); m.r0h = cellF("F.r0h", 0);
        for (int j = 0; j < 2; ++j) {
            m.du[j] = cellF("F.du%d", j); m.dw[j] = cellF("F.dw%d", j); m.dh[j] = cellF("F.dh%d", j);
        }
        m.x = cellF("F.x", 0); m.p0 = cellF("F.p0", 0); m.p1 = cellF("F.p1", 0); m.q = cellF("F.q", 0);
        const double rt = c->mp_rtol != 0.0 ? c->mp_rtol : kMixedRtol;
        m.tol2 = rt * rt;
        for (size_t lv = 0; lv < lg.size(); ++lv) {
            const Geom &g = lg[lv];
            const int l_ = (int)lv;
            LevelF l;
            l.G = g;
            auto la = [&](const char *fmt) { return (float *)arr(g, g.nz, g.nx, 4, fmt, l_); };
            l.c = la("F.L%d.c"); l.d = la("F.L%d.d"); l.wd = la("F.L%d.wd");
            l.ax = (float *)arr(g, g.nz, g.nx + 1, 4, "F.L%d.ax", l_);
            l.az = (float *)arr(g, g.nz + 1, g.nx, 4, "F.L%d.az", l_);
            l.r = la("F.L%d.r"); l.e = la("F.L%d.e"); l.e2 = la("F.L%d.e2"); l.r_alt = la("F.L%d.r_alt");
            ctx->Lf.push_back(l);
        }
    }
    // group counters of the grid sums, then two buffers of 4 x (blocks <=
    // tiles) partials for the persistent kernels (or a grid sum's block and
    // group totals)
    ctx->partials = take(round_up((kGcntDoubles + 8 * nb_all) * sizeof(double), 256));
    ctx->sc = (Scal *)take(round_up(sizeof(Scal), 256));
    if ((size_t)(ptr - ctx->mem) > total) {
        gea_destroy(ctx);
        return GEA_ERR_NOMEM;
    }
    {
        // g z of the cell centres z_k = (k + 1/2) dz and of the z-faces k dz
        std::vector<double> h(2 * (size_t)G.nz + 1);
        for (int k = 0; k < G.nz; ++k) h[k] = ctx->F.g * ((k + 0.5) * G.dz);
        for (int k = 0; k <= G.nz; ++k) h[G.nz + k] = ctx->F.g * (k * G.dz);
        if (cudaMemcpy(ctx->gzc, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            gea_destroy(ctx);
            return GEA_ERR_CUDA;
        }
    }
    if (dbg) {
        // the region table on the device, two check results, then the poison
        std::vector<PadRegionDev> hr;
        for (const gea_pad_region &pr : ctx->pads)
            hr.push_back(PadRegionDev{(char *)pr.ptr, (long long)pr.span, pr.elem_bytes, pr.pitch, pr.rows, pr.cols});
        if (cudaMalloc(&ctx->dpads, hr.size() * sizeof(PadRegionDev)) != cudaSuccess ||
            cudaMalloc(&ctx->dpres, 2 * sizeof(PadResult)) != cudaSuccess) {
            cudaGetLastError();
            gea_destroy(ctx);
            return GEA_ERR_NOMEM;
        }
        if (cudaMemcpy(ctx->dpads, hr.data(), hr.size() * sizeof(PadRegionDev), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            launch_pad_poison(ctx->dpads, (int)hr.size(), 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            gea_destroy(ctx);
            return GEA_ERR_CUDA;
        }
    }
    for (int e = 0; e < 8; ++e) cudaEventCreate(&ctx->ev[e]);
    ctx->nev = 8;
    // step driver: the persistent kernel pays off while a phase is a few
    // tiles per resident block (its phases are latency-bound); on larger
    // grids the per-phase kernels keep more blocks resident per SM
    if (!(c->flags & (GEA_FLAG_GRAPH | GEA_FLAG_KEEP_R0))) {
        const PersistOps &o = persist_ops(ctx->shape);
        const int pmax = ctx->mixed ? o.mixed_max_blocks() : o.max_blocks();
        cudaGetLastError();
        if (pmax > 0 && (long long)nb <= (long long)kPersistTilesPerBlock * pmax)
            ctx->pers_blocks = pmax < (int)nb ? pmax : (int)nb;
    }
    if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        gea_destroy(ctx);
        return GEA_ERR_CUDA;
    }
    *out = ctx;
    return GEA_OK;
}

int gea_set_stream(gea_ctx *ctx, void *stream)
{
    if (!ctx) return GEA_ERR_INVAL;
    ctx->stream = (cudaStream_t)stream;
    return GEA_OK;
}

int gea_set_state(gea_ctx *ctx, const gea_state_view *v)
{
    if (!ctx || !v) return GEA_ERR_INVAL;
    const Geom &G = ctx->G;
    const int nx = G.nx, nz = G.nz;
    if (!v->rho) return fail(ctx, GEA_ERR_INVAL, "rho is null");
    State &S = ctx->S[0];
    const double *src[11] = {v->rho, v->u, v->w, v->T, v->h, v->p, v->pp, v->pold, v->phix, v->phiz,
                             v->Kold};
    double *dst[11] = {S.rho, S.u, S.w, S.T, S.h, S.p, S.pp, S.pold, S.phix, S.phiz, S.Kold};
    // K^{n-1} belongs to the state only in the literal reading of eq. step3_sd
    const int nf = ctx->F.k_lagged ? 11 : 10;
    // arguments are checked before the context is touched
    if (v->kind == GEA_STATE_CONSERVATIVE) {
        if (!v->rhou || !v->rhow || !v->rhoe) return fail(ctx, GEA_ERR_INVAL, "null conservative field");
    } else if (v->kind == GEA_STATE_FULL) {
        for (int f = 0; f < nf; ++f)
            if (!src[f]) return fail(ctx, GEA_ERR_INVAL, "null field %d", f);
    } else {
        return fail(ctx, GEA_ERR_INVAL, "unknown state kind %d", v->kind);
    }
    // from here the old state is being replaced: until this call succeeds
    // the context holds none
    ctx->have_state = false;
    // reset the device scalars: status, counters, step count
    CK(cudaMemsetAsync(ctx->sc, 0, sizeof(Scal), ctx->stream));
    if (v->kind == GEA_STATE_CONSERVATIVE) {
        const size_t cellw = ctx->stage_stride;
        double *st = ctx->stage;
        int rc;
        if ((rc = copy_in(ctx, st, v->rho, nx, nz)) || (rc = copy_in(ctx, st + cellw, v->rhou, nx, nz)) ||
            (rc = copy_in(ctx, st + 2 * cellw, v->rhow, nx, nz)) ||
            (rc = copy_in(ctx, st + 3 * cellw, v->rhoe, nx, nz)))
            return rc;
        launch_derive(G, ctx->F, st, st + cellw, st + 2 * cellw, st + 3 * cellw, S, ctx->sc, ctx->stream);
        CK(cudaGetLastError());
    } else {
        for (int f = 0; f < nf; ++f) {
            const int cols = f == 8 ? nx + 1 : nx, rows = f == 9 ? nz + 1 : nz;
            int rc = copy_in(ctx, dst[f], src[f], cols, rows);
            if (rc) return rc;
        }
    }
    if (v->kind == GEA_STATE_FULL) {
        // a full state is taken as given (only the derivation from the
        // conservative fields checks rho and T): no round trip to the device
        ctx->base = 0;
        ctx->steps_at_sync = 0;
        ctx->have_state = true;
        return GEA_OK;
    }
    Scal h;
    int rc = read_scal(ctx, &h);
    if (rc) return rc;
    if (h.bad_cells) {
        ctx->have_state = false;
        return fail(ctx, GEA_ERR_INVAL, "%d cells with rho <= 0 or T <= 0", h.bad_cells);
    }
    ctx->base = 0;
    ctx->steps_at_sync = 0;
    ctx->have_state = true;
    return GEA_OK;
}

namespace {
// NVTX range around the enqueueing of steps (the host side of gea_step)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

int gea_step_async(gea_ctx *ctx, int32_t n)
{
    if (!ctx || n < 0) return GEA_ERR_INVAL;
    NvtxRange range(ctx->pers_blocks > 0 && !ctx->net ? "gea_step persistent" : "gea_step graph");
    if (!ctx->have_state) return fail(ctx, GEA_ERR_STATE, "no state set");
    if (n == 0) return GEA_OK;
    if (ctx->pers_blocks > 0 && !ctx->net) {
        StepArgs a[2] = {step_args(ctx, 0), step_args(ctx, 1)};
        const int first = (int)((ctx->base + ctx->steps_at_sync) & 1);
        const PersistOps &o = persist_ops(ctx->shape);
        if (ctx->mixed)
            CK(o.launch_mixed(a, ctx->L[0], ctx->mx, ctx->Lf.data(), (int)ctx->Lf.size(), kCoarseSweeps,
                                       ctx->C.n_corr, ctx->C.jac_maxit, ctx->C.cg_maxit, first, n,
                                       ctx->pers_blocks, ctx->wait_polls, ctx->stream));
        else
            CK(o.launch(a, ctx->L.data(), (int)ctx->L.size(), kCoarseSweeps, ctx->C.n_corr,
                                 ctx->C.jac_maxit, ctx->C.cg_maxit, first, n, ctx->pers_blocks,
                                 ctx->wait_polls, ctx->stream));
        ctx->steps_at_sync += n;
        return GEA_OK;
    }
    int rc = ensure_graphs(ctx);
    if (rc) return rc;
    // the slot holding the newest state is base + steps launched so far;
    // launches alternate the two graphs
    for (int s = 0; s < n; ++s) {
        const int from = (int)((ctx->base + ctx->steps_at_sync) & 1);
        CK(cudaGraphLaunch(ctx->exec[from], ctx->stream));
        ctx->steps_at_sync += 1;
    }
    return GEA_OK;
}

int gea_sync(gea_ctx *ctx)
{
    if (!ctx) return GEA_ERR_INVAL;
    Scal h;
    int rc = read_scal(ctx, &h);
    if (rc) return rc;
    // steps that did not complete (after a device-side error) did not move
    // the state
    ctx->steps_at_sync = h.steps_done;
    if (h.last_status == GEA_ERR_NOCONV) return fail(ctx, GEA_ERR_NOCONV, "a linear solve reached its iteration cap");
    if (h.last_status == GEA_ERR_NONFINITE) return fail(ctx, GEA_ERR_NONFINITE, "non-finite residual");
    if (h.last_status) return fail(ctx, h.last_status, "device status %d", h.last_status);
    return GEA_OK;
}

int gea_step(gea_ctx *ctx, int32_t n)
{
    int rc = gea_step_async(ctx, n);
    if (rc) return rc;
    return gea_sync(ctx);
}

int gea_get_state(gea_ctx *ctx, gea_state_view *v)
{
    if (!ctx || !v) return GEA_ERR_INVAL;
    if (!ctx->have_state) return fail(ctx, GEA_ERR_STATE, "no state set");
    Scal h;
    int rc = read_scal(ctx, &h);
    if (rc) return rc;
    const Geom &G = ctx->G;
    const int nx = G.nx, nz = G.nz;
    const State &S = ctx->S[current_slot(ctx, h)];
    if (v->kind == GEA_STATE_FULL) {
        double *dst[11] = {v->rho, v->u, v->w, v->T, v->h, v->p, v->pp, v->pold, v->phix, v->phiz, v->Kold};
        const double *src[11] = {S.rho, S.u, S.w, S.T, S.h, S.p, S.pp, S.pold, S.phix, S.phiz, S.Kold};
        const int nf = ctx->F.k_lagged ? 11 : 10;
        for (int f = 0; f < nf; ++f) {
            if (!dst[f]) continue;
            const int cols = f == 8 ? nx + 1 : nx, rows = f == 9 ? nz + 1 : nz;
            if ((rc = copy_out(ctx, dst[f], src[f], cols, rows))) return rc;
        }
    } else if (v->kind == GEA_STATE_CONSERVATIVE) {
        // computed on the device into the staging area, then copied out
        const size_t cellw = ctx->stage_stride;
        double *st = ctx->stage;
        launch_conserve(G, ctx->F, S, st, st + cellw, st + 2 * cellw, st + 3 * cellw, ctx->stream);
        CK(cudaGetLastError());
        double *dst[4] = {v->rho, v->rhou, v->rhow, v->rhoe};
        for (int f = 0; f < 4; ++f) {
            if (!dst[f]) continue;
            if ((rc = copy_out(ctx, dst[f], st + f * cellw, nx, nz))) return rc;
        }
    } else {
        return fail(ctx, GEA_ERR_INVAL, "unknown state kind %d", v->kind);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return GEA_OK;
}

int gea_get_diag(gea_ctx *ctx, const double *theta_bar, double *theta_prime, double *mass,
                 double *energy)
{
    if (!ctx) return GEA_ERR_INVAL;
    if (!ctx->have_state) return fail(ctx, GEA_ERR_STATE, "no state set");
    Scal h;
    int rc = read_scal(ctx, &h);
    if (rc) return rc;
    const Geom &G = ctx->G;
    if (theta_prime && !theta_bar) return fail(ctx, GEA_ERR_INVAL, "theta_prime needs theta_bar");
    if (theta_bar)
        CK(cudaMemcpyAsync(ctx->thbar, theta_bar, G.nz * sizeof(double), cudaMemcpyDefault, ctx->stream));
    launch_diag(G, ctx->F, ctx->S[current_slot(ctx, h)], ctx->thbar, theta_prime ? ctx->thout : nullptr,
                ctx->sc, ctx->partials, ctx->stream);
    CK(cudaGetLastError());
    if (theta_prime && (rc = copy_out(ctx, theta_prime, ctx->thout, G.nx, G.nz))) return rc;
    if ((rc = read_scal(ctx, &h))) return rc;
    if (mass) *mass = h.mass;
    if (energy) *energy = h.energy;
    return GEA_OK;
}

int gea_get_stats(gea_ctx *ctx, gea_stats *s)
{
    if (!ctx || !s) return GEA_ERR_INVAL;
    Scal h;
    int rc = read_scal(ctx, &h);
    if (rc) return rc;
    memset(s, 0, sizeof(*s));
    s->steps_done = h.steps_done;
    s->jac_u = h.last_sweeps[0];
    s->jac_h = h.last_sweeps[1];
    for (int c = 0; c < 4; ++c) {
        s->cg_iters[c] = h.last_cg_iters[c];
        s->cg_relres[c] = h.last_cg_relres[c];
    }
    s->status = h.last_status;
    s->mg_levels = ctx->mixed ? (int)ctx->Lf.size() : (int)ctx->L.size();
    s->launches = h.launches;
    const bool pers = ctx->pers_blocks > 0 && !ctx->net;
    s->driver = ctx->mixed ? (pers ? 3 : 2) : pers ? 1 : 0;
    return GEA_OK;
}

int gea_get_field(gea_ctx *ctx, int32_t which, double *host)
{
    if (!ctx || !host) return GEA_ERR_INVAL;
    const Geom &G = ctx->G;
    Scal h;
    if (int rc0 = read_scal(ctx, &h)) return rc0;
    const bool slot_u1 = h.u1_slot != 0, slot_h1 = h.h1_slot != 0;
    const double *src = nullptr;
    int cols = G.nx, rows = G.nz;
    switch (which) {
    case GEA_FIELD_RHO1: src = ctx->rho1; break;
    case GEA_FIELD_U1: src = slot_u1 ? ctx->ub : ctx->ua; break;
    case GEA_FIELD_W1: src = slot_u1 ? ctx->wb : ctx->wa; break;
    case GEA_FIELD_H1:
        // mixed precision: h^{n+1} = h^n + dh goes straight into the new state
        src = ctx->mixed ? ctx->S[current_slot(ctx, h)].h : slot_h1 ? ctx->hb : ctx->ha;
        break;
    case GEA_FIELD_RHO2: src = ctx->rho2; break;
    case GEA_FIELD_HX: src = ctx->Hx; break;
    case GEA_FIELD_HZ: src = ctx->Hz; break;
    case GEA_FIELD_B: src = ctx->b; break;
    case GEA_FIELD_DX: src = ctx->Dx; cols = G.nx + 1; break;
    case GEA_FIELD_DZ: src = ctx->Dz; rows = G.nz + 1; break;
    case GEA_FIELD_HC: src = ctx->L[0].c; break;
    case GEA_FIELD_HAX: src = ctx->L[0].ax; cols = G.nx + 1; break;
    case GEA_FIELD_HAZ: src = ctx->L[0].az; rows = G.nz + 1; break;
    case GEA_FIELD_R0:
        if (!ctx->r0keep) return fail(ctx, GEA_ERR_INVAL, "R0 needs GEA_FLAG_KEEP_R0");
        src = ctx->r0keep;
        break;
    default: return fail(ctx, GEA_ERR_INVAL, "unknown field %d", which);
    }
    int rc = copy_out(ctx, host, src, cols, rows);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return GEA_OK;
}

double gea_last_pressure_ms(gea_ctx *ctx)
{
    if (!ctx) return -1.0;
    if (ctx->pers_blocks > 0 && !ctx->net) {
        Scal h;
        if (read_scal(ctx, &h)) return -1.0;
        return (double)h.press_ns * 1e-6;
    }
    if (!ctx->exec[0]) return -1.0;
    double tot = 0.0;
    for (int c = 0; c < ctx->C.n_corr; ++c) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev[2 * c], ctx->ev[2 * c + 1]) != cudaSuccess) {
            cudaGetLastError();
            return -1.0;
        }
        tot += ms;
    }
    return tot;
}

int gea_profile_step(gea_ctx *ctx, gea_kernel_time *out, int32_t max_entries, int32_t *n_entries)
{
    if (!ctx || (!out && max_entries > 0) || !n_entries) return GEA_ERR_INVAL;
    if (!ctx->have_state) return fail(ctx, GEA_ERR_STATE, "no state set");
    Scal h;
    int rc = read_scal(ctx, &h);
    if (rc) return rc;
    if (h.status) return fail(ctx, h.status, "device status %d", h.status);
    const int from = current_slot(ctx, h);
    EventTracer tr(ctx->sc);
    rc = record_any(ctx, from, ctx->stream, false, &tr);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<gea_kernel_time> agg;
    for (auto &r : tr.recs) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.e0, r.e1));
        size_t j = 0;
        for (; j < agg.size(); ++j)
            if (!strcmp(agg[j].name, r.name)) break;
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
    ctx->steps_at_sync += 1;
    return gea_sync(ctx);
}

namespace {

int pad_reset(gea_ctx *ctx)
{
    PadResult h[2];
    for (PadResult &r : h) {
        r.bad = 0;
        r.key = ~0ull;
        r.first = INT_MAX;
        r.pad_ = 0;
    }
    CK(cudaMemcpyAsync(ctx->dpres, h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    return GEA_OK;
}

// rep from the per-launch tracking (slot 0, names: the launches) and the
// final count (slot 1)
int pad_report(gea_ctx *ctx, const std::vector<const char *> *names, gea_pad_report *rep)
{
    PadResult h[2];
    CK(cudaMemcpyAsync(h, ctx->dpres, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    memset(rep, 0, sizeof(*rep));
    rep->bad = (int64_t)h[1].bad;
    rep->launch = -1;
    const PadResult &f = names ? h[0] : h[1];
    if (names && f.first != INT_MAX) {
        rep->launch = f.first;
        if (f.first >= 0 && (size_t)f.first < names->size())
            snprintf(rep->kernel, sizeof(rep->kernel), "%s", (*names)[f.first]);
    }
    if (f.key != ~0ull) {
        const size_t reg = (size_t)(f.key >> 40);
        const long long e = (long long)(f.key & ((1ull << 40) - 1));
        if (reg < ctx->pads.size()) {
            const gea_pad_region &pr = ctx->pads[reg];
            snprintf(rep->array, sizeof(rep->array), "%s", pr.name);
            rep->row = (int32_t)(e / pr.pitch);
            rep->col = (int32_t)(e % pr.pitch);
        }
    }
    return GEA_OK;
}

}  // namespace

int gea_debug_pad_regions(gea_ctx *ctx, gea_pad_region *out, int32_t max, int32_t *n)
{
    if (!ctx || !n || (!out && max > 0)) return GEA_ERR_INVAL;
    if (!ctx->dpads) return fail(ctx, GEA_ERR_INVAL, "the context was created without GEA_FLAG_DEBUG_PADS");
    *n = (int32_t)ctx->pads.size();
    for (size_t j = 0; j < ctx->pads.size() && (int32_t)j < max; ++j) out[j] = ctx->pads[j];
    return GEA_OK;
}

int gea_debug_poison(gea_ctx *ctx)
{
    if (!ctx) return GEA_ERR_INVAL;
    if (!ctx->dpads) return fail(ctx, GEA_ERR_INVAL, "the context was created without GEA_FLAG_DEBUG_PADS");
    CK(launch_pad_poison(ctx->dpads, (int)ctx->pads.size(), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GEA_OK;
}

int gea_debug_check_pads(gea_ctx *ctx, gea_pad_report *rep)
{
    if (!ctx || !rep) return GEA_ERR_INVAL;
    if (!ctx->dpads) return fail(ctx, GEA_ERR_INVAL, "the context was created without GEA_FLAG_DEBUG_PADS");
    int rc = pad_reset(ctx);
    if (rc) return rc;
    CK(launch_pad_check(ctx->dpads, (int)ctx->pads.size(), ctx->dpres + 1, 0, ctx->stream));
    return pad_report(ctx, nullptr, rep);
}

int gea_debug_step(gea_ctx *ctx, gea_pad_report *rep)
{
    if (!ctx || !rep) return GEA_ERR_INVAL;
    if (!ctx->dpads) return fail(ctx, GEA_ERR_INVAL, "the context was created without GEA_FLAG_DEBUG_PADS");
    if (!ctx->have_state) return fail(ctx, GEA_ERR_STATE, "no state set");
    Scal h;
    int rc = read_scal(ctx, &h);
    if (rc) return rc;
    if (h.status) return fail(ctx, h.status, "device status %d", h.status);
    if ((rc = pad_reset(ctx))) return rc;
    const int from = current_slot(ctx, h);
    PadTracer tr(ctx);
    rc = record_any(ctx, from, ctx->stream, false, &tr);
    if (rc) return rc;
    CK(tr.err);
    CK(launch_pad_check(ctx->dpads, (int)ctx->pads.size(), ctx->dpres + 1, INT_MAX, ctx->stream));
    if ((rc = pad_report(ctx, &tr.names, rep))) return rc;
    ctx->steps_at_sync += 1;
    return gea_sync(ctx);
}

int gea_set_tiles_per_block(gea_ctx *ctx, int32_t n)
{
    if (!ctx || n < 0 || n > kMaxTilesPerBlock) return GEA_ERR_INVAL;
    if (ctx->stream) CK(cudaStreamSynchronize(ctx->stream));
    // the step graphs hold the launch shapes
    for (int f = 0; f < 2; ++f) {
        if (ctx->exec[f]) cudaGraphExecDestroy(ctx->exec[f]);
        if (ctx->graph[f]) cudaGraphDestroy(ctx->graph[f]);
        ctx->exec[f] = nullptr;
        ctx->graph[f] = nullptr;
    }
    ctx->tiles_per_block = n;
    return GEA_OK;
}

int gea_set_smoother_weight(gea_ctx *ctx, double omega)
{
    if (!ctx || !(omega > 0.0) || !(omega < 2.0)) return GEA_ERR_INVAL;
    if (ctx->stream) CK(cudaStreamSynchronize(ctx->stream));
    // the step graphs hold the physical constants of their kernels
    for (int f = 0; f < 2; ++f) {
        if (ctx->exec[f]) cudaGraphExecDestroy(ctx->exec[f]);
        if (ctx->graph[f]) cudaGraphDestroy(ctx->graph[f]);
        ctx->exec[f] = nullptr;
        ctx->graph[f] = nullptr;
    }
    ctx->F.omega = omega;
    return GEA_OK;
}

int gea_apply_precond(gea_ctx *ctx, const double *r, double *z)
{
    if (!ctx || !r || !z) return GEA_ERR_INVAL;
    if (ctx->mixed) return fail(ctx, GEA_ERR_INVAL, "the FP64 preconditioner of a mixed-precision context is not kept");
    if (!ctx->have_state) return fail(ctx, GEA_ERR_STATE, "no state set");
    Scal h;
    int rc = read_scal(ctx, &h);
    if (rc) return rc;
    if (h.steps_done < 1) return fail(ctx, GEA_ERR_STATE, "no completed step: the operator is not assembled");
    // the V-cycle kernels run while the CG loop is open; their reduction
    // (r.z) writes the loop scalars, which are put back afterwards
    Scal run = h;
    run.done[LOOP_CG] = 0;
    run.status = 0;
    run.cg_it = 0;
    CK(cudaMemcpyAsync(ctx->sc, &run, sizeof(Scal), cudaMemcpyHostToDevice, ctx->stream));
    Level *L = ctx->L.data();
    rc = copy_in(ctx, L[0].r, r, ctx->G.nx, ctx->G.nz);
    if (!rc) {
        StepArgs a = step_args(ctx, 0);
        launch_vcycle(a, L, (int)ctx->L.size(), kCoarseSweeps, ctx->stream, nullptr);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = fail(ctx, GEA_ERR_CUDA, "V-cycle launch: %s", cudaGetErrorString(e));
    }
    if (!rc) rc = copy_out(ctx, z, L[0].e2, ctx->G.nx, ctx->G.nz);
    // the scalars of the last completed step go back, also after an error
    CK(cudaMemcpyAsync(ctx->sc, &h, sizeof(Scal), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return rc;
}

int gea_set_tile_shape(gea_ctx *ctx, int32_t shape)
{
    if (!ctx || shape < 0 || shape >= NSHAPES) return GEA_ERR_INVAL;
    if (ctx->stream) CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->pers_blocks > 0) {
        // the persistent driver stays; its grid follows the shape's occupancy
        // and tile count
        const PersistOps &o = persist_ops(shape);
        const int pmax = ctx->mixed ? o.mixed_max_blocks() : o.max_blocks();
        cudaGetLastError();
        if (pmax <= 0) return fail(ctx, GEA_ERR_CUDA, "no resident blocks for tile shape %d", shape);
        const long long nt = shape_tiles(ctx->G, o.bx, o.bz);
        ctx->pers_blocks = (long long)pmax < nt ? pmax : (int)nt;
    }
    ctx->shape = shape;
    // a phase trace was sized for the previous grid of blocks
    ctx->trace = nullptr;
    ctx->trace_bars = 0;
    return GEA_OK;
}

int gea_set_wait_limit(gea_ctx *ctx, int64_t polls)
{
    if (!ctx) return GEA_ERR_INVAL;
    // a limit can only be lowered: above the default the wait stays bounded
    // by the default
    ctx->wait_polls = polls < 0 ? -1 : polls > (int64_t)kSpinLimit ? (int64_t)kSpinLimit : polls;
    return GEA_OK;
}

int gea_set_trace(gea_ctx *ctx, uint64_t *trace, int32_t max_barriers, int64_t capacity, int32_t *blocks)
{
    if (!ctx || max_barriers < 0 || (trace && max_barriers == 0)) return GEA_ERR_INVAL;
    if (blocks) *blocks = ctx->pers_blocks;
    if (!trace) {
        ctx->trace = nullptr;
        ctx->trace_bars = 0;
        return GEA_OK;
    }
    if (ctx->pers_blocks <= 0)
        return fail(ctx, GEA_ERR_INVAL, "the phase trace needs the persistent driver");
    if (capacity < 2LL * (max_barriers + 1) * ctx->pers_blocks)
        return fail(ctx, GEA_ERR_INVAL, "trace buffer of %lld values holds fewer than 2 x %d x %d",
                    (long long)capacity, max_barriers + 1, ctx->pers_blocks);
    if (reinterpret_cast<uintptr_t>(trace) % 8) return fail(ctx, GEA_ERR_INVAL, "trace buffer not 8-byte aligned");
    ctx->trace = reinterpret_cast<unsigned long long *>(trace);
    ctx->trace_bars = max_barriers;
    return GEA_OK;
}

int gea_attach_net(gea_ctx *ctx, gea_net *net, int32_t mode)
{
    if (!ctx || mode < 0 || mode > 3 || (mode != 0 && !net)) return GEA_ERR_INVAL;
    const Geom &G = ctx->G;
    if ((mode & 2) && ctx->mixed)
        return fail(ctx, GEA_ERR_INVAL, "the network preconditioner is for the FP64 step (mode 2 and 3)");
    if (mode != 0 && (G.nx % 8 || G.nz % 8 || !gea_net_fits(net, 1, G.nz, G.nx)))
        return fail(ctx, GEA_ERR_INVAL, "grid %d x %d does not fit the network", G.nx, G.nz);
    if (ctx->stream) CK(cudaStreamSynchronize(ctx->stream));
    // the step graphs change
    for (int f = 0; f < 2; ++f) {
        if (ctx->exec[f]) cudaGraphExecDestroy(ctx->exec[f]);
        if (ctx->graph[f]) cudaGraphDestroy(ctx->graph[f]);
        ctx->exec[f] = nullptr;
        ctx->graph[f] = nullptr;
    }
    if (ctx->net_r) cudaFree(ctx->net_r);
    if (ctx->net_e) cudaFree(ctx->net_e);
    if (ctx->net_s) cudaFree(ctx->net_s);
    ctx->net_r = ctx->net_e = nullptr;
    ctx->net_s = nullptr;
    ctx->net = nullptr;
    ctx->net_mode = 0;
    if (mode == 0) return GEA_OK;
    const size_t bytes = (size_t)G.nx * G.nz * sizeof(float);
    if (cudaMalloc(&ctx->net_r, bytes) != cudaSuccess || cudaMalloc(&ctx->net_e, bytes) != cudaSuccess ||
        ((mode & 2) && cudaMalloc(&ctx->net_s, arr_bytes(G, G.nz)) != cudaSuccess)) {
        cudaGetLastError();
        if (ctx->net_r) cudaFree(ctx->net_r);
        if (ctx->net_e) cudaFree(ctx->net_e);
        ctx->net_r = ctx->net_e = nullptr;
        ctx->net_s = nullptr;
        return fail(ctx, GEA_ERR_NOMEM, "network buffers");
    }
    if (ctx->net_s) CK(cudaMemsetAsync(ctx->net_s, 0, arr_bytes(G, G.nz), ctx->stream));
    // one eager forward pass outside any capture sets up the network's
    // kernels (launch attributes are set on first use)
    CK(cudaMemsetAsync(ctx->net_r, 0, bytes, ctx->stream));
    if (gea_net_run(net, ctx->stream, 1, G.nz, G.nx, ctx->net_r, ctx->net_e) < 0)
        return fail(ctx, GEA_ERR_CUDA, "network forward failed");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->net = net;
    ctx->net_mode = mode;
    return GEA_OK;
}

}  // extern "C"

struct gea_ensemble {
    std::vector<gea_ctx *> m;
    std::vector<int> groups;         // group table of the launch (PersistOps::launch_ensemble)
    int ngroups = 0;
    std::vector<int> nbm;            // blocks each member runs on (1: a block it may share)
    int blocks = 0;
    cudaStream_t st = nullptr;
    size_t argb = 0;                 // bytes of one member's argument block
    char *hargs = nullptr;           // pinned host staging of the argument blocks
    void *dargs = nullptr;
    int *dgroups = nullptr;
    int shape = SHAPE_32x8;          // the members' tile shape
    bool mixed = false;              // mixed-precision members (GEA_FLAG_MIXED)
    // the launch as a CUDA graph: one instantiated graph (a cooperative kernel
    // node reading its own device copy of the argument blocks) per state slot
    // parity and step count, used while every member is at the same parity
    bool use_graph = true;
    cudaStream_t cap = nullptr;      // private stream for the capture
    struct Graph {
        int parity, n;
        // the members' settings that the argument blocks carry, when built:
        // barrier poll limits and smoother weights
        std::vector<long long> polls;
        std::vector<double> omegas;
        void *dargs;
        cudaGraph_t g;
        cudaGraphExec_t x;
    };
    std::vector<Graph> graphs;
};

namespace {

// fill the host staging with every member's argument block
void ensemble_fill(gea_ensemble *e, int n, int parity)
{
    for (size_t i = 0; i < e->m.size(); ++i) {
        gea_ctx *c = e->m[i];
        StepArgs a[2] = {step_args(c, 0), step_args(c, 1)};
        const int first = parity >= 0 ? parity : (int)((c->base + c->steps_at_sync) & 1);
        if (e->mixed)
            persist_args_fill_mixed(e->hargs + i * e->argb, a, c->L[0], c->mx, c->Lf.data(), (int)c->Lf.size(),
                                    kCoarseSweeps, c->C.n_corr, c->C.jac_maxit, c->C.cg_maxit, first, n,
                                    c->wait_polls);
        else
            persist_args_fill(e->hargs + i * e->argb, a, c->L.data(), (int)c->L.size(), kCoarseSweeps,
                              c->C.n_corr, c->C.jac_maxit, c->C.cg_maxit, first, n, c->wait_polls);
    }
}

// the graph of n steps from state slot `parity` with the members' current
// settings, built on first use
gea_ensemble::Graph *ensemble_graph(gea_ensemble *e, int n, int parity)
{
    std::vector<long long> polls;
    std::vector<double> omegas;
    for (gea_ctx *c : e->m) {
        polls.push_back(c->wait_polls);
        omegas.push_back(c->F.omega);
    }
    for (auto &g : e->graphs)
        if (g.parity == parity && g.n == n && g.polls == polls && g.omegas == omegas) return &g;
    gea_ensemble::Graph g{parity, n, polls, omegas, nullptr, nullptr, nullptr};
    const size_t bytes = e->argb * e->m.size();
    if (cudaStreamSynchronize(e->st) != cudaSuccess || cudaMalloc(&g.dargs, bytes) != cudaSuccess) return nullptr;
    ensemble_fill(e, n, parity);
    bool ok = cudaMemcpy(g.dargs, e->hargs, bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        const cudaError_t le = persist_ops(e->shape).launch_ensemble(g.dargs, e->mixed ? 1 : 0, e->dgroups,
                                                                    e->ngroups, e->blocks, e->cap);
        const cudaError_t ce = cudaStreamEndCapture(e->cap, &g.g);
        ok = le == cudaSuccess && ce == cudaSuccess && g.g &&
             cudaGraphInstantiate(&g.x, g.g, 0) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        if (g.g) cudaGraphDestroy(g.g);
        cudaFree(g.dargs);
        return nullptr;
    }
    e->graphs.push_back(std::move(g));
    return &e->graphs.back();
}

// Blocks of an ensemble launch for members of weights wt (tiles[i] tiles
// each) on B co-resident blocks, as a group table (PersistOps::
// launch_ensemble) and the blocks each member runs on. A member whose share
// B wt / sum(wt) is below one block runs on a block it shares with other
// such members, packed in member order while their shares add up to at most
// one block (they run in turn); the others split the remaining blocks in
// proportion to their weights (at least one each, at most one per tile, the
// remainder by largest fractional share). If that would leave a member
// without a block, every member gets a block of its own (n <= B) and the
// rest in proportion. Returns false if no partition fits.
bool ensemble_partition(const std::vector<double> &wt, const std::vector<long long> &tiles, int B,
                        std::vector<int> &groups, int &ngroups, std::vector<int> &nbm, int &blocks)
{
    const int n = (int)wt.size();
    auto split = [&](const std::vector<int> &who, int avail, std::vector<int> &nb) -> bool {
        nb.assign(who.size(), 1);
        if ((int)who.size() > avail) return false;
        double tot = 0.0;
        for (int i : who) tot += wt[i];
        const int extra = avail - (int)who.size();
        std::vector<double> frac(who.size(), 0.0);
        int used = (int)who.size();
        for (size_t k = 0; k < who.size(); ++k) {
            const double share = (double)extra * wt[who[k]] / tot;
            int e = (int)share;
            if (e > tiles[who[k]] - 1) e = (int)tiles[who[k]] - 1;
            nb[k] += e;
            used += e;
            frac[k] = share - e;
        }
        while (used < avail) {
            int best = -1;
            for (size_t k = 0; k < who.size(); ++k)
                if (nb[k] < tiles[who[k]] && (best < 0 || frac[k] > frac[best])) best = (int)k;
            if (best < 0) break;
            nb[best] += 1;
            frac[best] = -1.0;
            used += 1;
        }
        return true;
    };
    double tot = 0.0;
    for (double w : wt) tot += w;
    std::vector<int> big;
    std::vector<std::vector<int>> bins;
    double load = 2.0;
    for (int i = 0; i < n; ++i) {
        const double share = (double)B * wt[i] / tot;
        if (share >= 1.0) {
            big.push_back(i);
            continue;
        }
        if (load + share > 1.0) {
            bins.emplace_back();
            load = 0.0;
        }
        bins.back().push_back(i);
        load += share;
    }
    std::vector<int> nb;
    std::vector<int> gb{0}, gm{0}, order;
    nbm.assign(n, 1);
    if (split(big, B - (int)bins.size(), nb)) {
        for (size_t k = 0; k < big.size(); ++k) {
            gb.push_back(gb.back() + nb[k]);
            gm.push_back(gm.back() + 1);
            order.push_back(big[k]);
            nbm[big[k]] = nb[k];
        }
        for (const auto &bin : bins) {
            gb.push_back(gb.back() + 1);
            gm.push_back(gm.back() + (int)bin.size());
            order.insert(order.end(), bin.begin(), bin.end());
        }
    } else {
        std::vector<int> all(n);
        for (int i = 0; i < n; ++i) all[i] = i;
        if (!split(all, B, nb)) return false;
        gb.assign(1, 0);
        gm.assign(1, 0);
        order.clear();
        for (int i = 0; i < n; ++i) {
            gb.push_back(gb.back() + nb[i]);
            gm.push_back(gm.back() + 1);
            order.push_back(i);
            nbm[i] = nb[i];
        }
    }
    ngroups = (int)gb.size() - 1;
    blocks = gb.back();
    groups = gb;
    groups.insert(groups.end(), gm.begin(), gm.end());
    groups.insert(groups.end(), order.begin(), order.end());
    return true;
}

}  // namespace

extern "C" {

int gea_ensemble_create(gea_ctx **members, int32_t n, const double *weights, gea_ensemble **out)
{
    if (!members || n < 1 || !out) return GEA_ERR_INVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        gea_ctx *c = members[i];
        // all members FP64 or all mixed precision: one kernel per launch
        if (!c || c->net || c->r0keep || c->mixed != members[0]->mixed) return GEA_ERR_INVAL;
        for (int j = 0; j < i; ++j)
            if (members[j] == c) return GEA_ERR_INVAL;
    }
    // one launch, one block shape: the members' tile shape
    const int shape = members[0]->shape;
    for (int i = 1; i < n; ++i)
        if (members[i]->shape != shape) return GEA_ERR_INVAL;
    const PersistOps &ops = persist_ops(shape);
    const int B = ops.ensemble_max_blocks(members[0]->mixed ? 1 : 0);
    cudaGetLastError();
    if (B < 1) return GEA_ERR_INVAL;
    std::vector<long long> tiles(n);
    std::vector<double> wt(n);
    for (int i = 0; i < n; ++i) {
        tiles[i] = shape_tiles(members[i]->G, ops.bx, ops.bz);
        wt[i] = weights ? weights[i] : (double)tiles[i];
        if (!(wt[i] > 0.0) || !(wt[i] < 1e300)) return GEA_ERR_INVAL;
    }
    std::vector<int> groups, nbm;
    int ngroups = 0, blocks = 0;
    if (!ensemble_partition(wt, tiles, B, groups, ngroups, nbm, blocks)) return GEA_ERR_INVAL;
    gea_ensemble *e = new gea_ensemble();
    e->m.assign(members, members + n);
    e->groups = groups;
    e->ngroups = ngroups;
    e->nbm = nbm;
    e->blocks = blocks;
    e->shape = shape;
    e->mixed = members[0]->mixed;
    e->argb = persist_args_bytes(e->mixed ? 1 : 0);   // the kernel indexes an array of argument blocks
    e->st = members[0]->stream;
    if (cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&e->hargs, e->argb * n) != cudaSuccess ||
        cudaMalloc(&e->dargs, e->argb * n) != cudaSuccess ||
        cudaMalloc(&e->dgroups, sizeof(int) * groups.size()) != cudaSuccess ||
        cudaMemcpy(e->dgroups, groups.data(), sizeof(int) * groups.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        gea_ensemble_destroy(e);
        return GEA_ERR_NOMEM;
    }
    for (gea_ctx *c : e->m) c->stream = e->st;
    *out = e;
    return GEA_OK;
}

int gea_ensemble_plan(const double *weights, const int64_t *tiles, int32_t n, int32_t blocks,
                      int32_t *member_blocks, int32_t *member_group, int32_t *ngroups, int32_t *used_blocks)
{
    if (!weights || !tiles || n < 1 || blocks < 1 || !member_blocks || !member_group) return GEA_ERR_INVAL;
    std::vector<double> wt(weights, weights + n);
    std::vector<long long> tl(tiles, tiles + n);
    for (int i = 0; i < n; ++i)
        if (!(wt[i] > 0.0) || !(wt[i] < 1e300) || tl[i] < 1) return GEA_ERR_INVAL;
    std::vector<int> groups, nbm;
    int ng = 0, used = 0;
    if (!ensemble_partition(wt, tl, blocks, groups, ng, nbm, used)) return GEA_ERR_INVAL;
    const int *gm = groups.data() + ng + 1, *order = gm + ng + 1;
    for (int gi = 0; gi < ng; ++gi)
        for (int k = gm[gi]; k < gm[gi + 1]; ++k) member_group[order[k]] = gi;
    for (int i = 0; i < n; ++i) member_blocks[i] = nbm[i];
    if (ngroups) *ngroups = ng;
    if (used_blocks) *used_blocks = used;
    return GEA_OK;
}

int gea_ensemble_set_graph(gea_ensemble *e, int32_t on)
{
    if (!e) return GEA_ERR_INVAL;
    e->use_graph = on != 0;
    return GEA_OK;
}

int gea_ensemble_set_stream(gea_ensemble *e, void *stream)
{
    if (!e) return GEA_ERR_INVAL;
    if (e->st) cudaStreamSynchronize(e->st);
    e->st = (cudaStream_t)stream;
    for (gea_ctx *c : e->m) c->stream = e->st;
    return GEA_OK;
}

int gea_ensemble_blocks(const gea_ensemble *e, int32_t m)
{
    if (!e || m < 0 || m >= (int)e->m.size()) return -1;
    return e->nbm[m];
}

int gea_ensemble_step(gea_ensemble *e, int32_t n)
{
    if (!e || n < 0) return GEA_ERR_INVAL;
    if (n == 0) return GEA_OK;
    for (gea_ctx *c : e->m)
        if (!c->have_state) return GEA_ERR_STATE;
    int parity = -1;
    bool same = true;
    for (gea_ctx *c : e->m) {
        const int p = (int)((c->base + c->steps_at_sync) & 1);
        if (parity < 0) parity = p;
        else if (p != parity) same = false;
    }
    if (e->use_graph && same) {
        gea_ensemble::Graph *g = ensemble_graph(e, n, parity);
        if (g && cudaGraphLaunch(g->x, e->st) == cudaSuccess) {
            for (gea_ctx *c : e->m) c->steps_at_sync += n;
            return GEA_OK;
        }
        // no graph on this platform: launch directly from now on
        cudaGetLastError();
        e->use_graph = false;
    }
    // the staging buffer may still feed the previous launch's copy
    if (cudaStreamSynchronize(e->st) != cudaSuccess) return GEA_ERR_CUDA;
    ensemble_fill(e, n, -1);
    if (cudaMemcpyAsync(e->dargs, e->hargs, e->argb * e->m.size(), cudaMemcpyHostToDevice, e->st) !=
            cudaSuccess ||
        persist_ops(e->shape).launch_ensemble(e->dargs, e->mixed ? 1 : 0, e->dgroups, e->ngroups, e->blocks,
                                              e->st) != cudaSuccess) {
        cudaGetLastError();
        return GEA_ERR_CUDA;
    }
    for (gea_ctx *c : e->m) c->steps_at_sync += n;
    return GEA_OK;
}

int gea_ensemble_sync(gea_ensemble *e)
{
    if (!e) return GEA_ERR_INVAL;
    int first_err = GEA_OK;
    for (gea_ctx *c : e->m) {
        const int rc = gea_sync(c);
        if (rc && !first_err) first_err = rc;
    }
    return first_err;
}

void gea_ensemble_destroy(gea_ensemble *e)
{
    if (!e) return;
    if (e->st) cudaStreamSynchronize(e->st);
    else cudaDeviceSynchronize();
    for (auto &g : e->graphs) {
        cudaGraphExecDestroy(g.x);
        cudaGraphDestroy(g.g);
        cudaFree(g.dargs);
    }
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->hargs) cudaFreeHost(e->hargs);
    if (e->dargs) cudaFree(e->dargs);
    if (e->dgroups) cudaFree(e->dgroups);
    delete e;
}

const char *gea_last_error(const gea_ctx *ctx) { return ctx ? ctx->err : "null context"; }

void gea_destroy(gea_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (int f = 0; f < 2; ++f) {
        if (ctx->exec[f]) cudaGraphExecDestroy(ctx->exec[f]);
        if (ctx->graph[f]) cudaGraphDestroy(ctx->graph[f]);
    }
    for (int e = 0; e < ctx->nev; ++e) cudaEventDestroy(ctx->ev[e]);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->cap2) cudaStreamDestroy(ctx->cap2);
    if (ctx->mem) cudaFree(ctx->mem);
    if (ctx->dpads) cudaFree(ctx->dpads);
    if (ctx->dpres) cudaFree(ctx->dpres);
    if (ctx->net_r) cudaFree(ctx->net_r);
    if (ctx->net_e) cudaFree(ctx->net_e);
    if (ctx->net_s) cudaFree(ctx->net_s);
    delete ctx;
}

}  // extern "C"
