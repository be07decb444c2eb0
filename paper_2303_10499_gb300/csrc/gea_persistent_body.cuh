// gea_persistent_body.cuh -- n time steps of the GEA pressure-based Euler
// solver (Girfoglio, Quaini & Rozza, arXiv 2303.10499, Section 3) as one
// cooperative kernel.
//
// On grids of up to a few hundred thousand cells a step is a chain of ~90
// short phases, and launching each as its own kernel leaves the GPU waiting
// on launch latency. Here the blocks stay resident for the whole step: each
// phase is a block-stride loop over tiles running the tile functions of
// gea_tiles_body.cuh, phases are separated by a grid barrier, and every
// residual norm or CG dot product rides on the barrier: each block writes its
// partial before arriving and, once released, adds all the partials itself
// in a fixed order. The Jacobi and CG loops run inside the kernel; every
// block takes the same decisions because it computes the same totals, bit
// for bit, and updates its own copy of the loop scalars with them.
//
// The barrier waits spin on an acquire load with an iteration cap; a block
// that gives up sets GEA_ERR_TIMEOUT in the context status, and every block
// leaves the step at its next phase boundary when the status is set, so the
// kernel always ends.
//
// Like the tile functions, this file is included once per tile shape, inside
// that shape's namespace and after its tile functions (gea_persistent.cu:
// 32 x 8; gea_persistent_16x16.cu, gea_persistent_64x4.cu): the kernels run
// one thread per cell of a BX x BZ tile, and the shape's host entry points
// are collected in `ops` (PersistOps, gea_internal.cuh).

namespace {

// values per thread a grid reduction may carry: the block-sum scratch after
// the tile area holds kRedVals x NTHREADS doubles
constexpr int kRedVals = 4;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Arrival with acquire-release semantics: publishes this block's writes of
// the phase (ordered before it by the block barrier) and observes those of
// the blocks that arrived earlier.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}


__device__ __forceinline__ int rdi(const int *p) { return __ldcg(p); }

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int tid_of() { return threadIdx.x + threadIdx.y * BX; }

// The blocks that run one context's steps: this block's rank among them and
// their number (the whole grid for one context; a contiguous share of the
// grid per member in an ensemble launch), and the block's count of the
// barriers it has passed in this launch (shared memory; every block passes
// the same barriers).
struct Grp {
    int rank, nb;
    unsigned *gen;   // barriers this block has passed in this launch
    Scal *gs;        // the context's scalars in global memory (barrier words, status, results)
    unsigned long long spin_limit;   // polls of a barrier before the block gives up
    unsigned long long *trace;       // phase trace (null: off), see trace_entry
    int trace_bars;                  // barriers the trace holds
};

// Phase trace layout: 2 x nb values per row; row 0 holds each block's
// kernel entry time and SM, row k >= 1 each block's arrival at and release
// from the k-th grid barrier of the launch (%globaltimer, ns).
__device__ __forceinline__ void trace_entry(const Grp &g)
{
    if (g.trace && tid_of() == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        g.trace[2 * (size_t)g.rank] = globaltimer();
        g.trace[2 * (size_t)g.rank + 1] = smid;
    }
}

// The block's own copy of the context's scalars. Every block finishes every
// grid reduction itself (the same partials added in the same order give
// every block the same totals, bit for bit) and applies the same update to
// its copy, so the loop decisions (convergence flags, iteration counts, CG
// step lengths) are taken from shared memory, identically in every block.
// Block rank 0 publishes what the host reads.
__shared__ Scal s_ctl;

// Block-uniform stop flag, set by thread 0 at kernel entry and at the end of
// every grid barrier (the context's status, or an error of the block's own
// reductions), so that all threads of a block leave a step at the same
// phase boundary.
__shared__ int s_stop;

// Copy the context's scalars into the block's copy (all threads; kernel entry).
__device__ __forceinline__ void load_ctl(const Scal *gs)
{
    static_assert(sizeof(Scal) % 4 == 0, "Scal is copied as 32-bit words");
    const int *src = reinterpret_cast<const int *>(gs);
    int *dst = reinterpret_cast<int *>(&s_ctl);
    for (int w = tid_of(); w < (int)(sizeof(Scal) / 4); w += NTHREADS) dst[w] = __ldcg(&src[w]);
}

// Grid barrier on a monotone arrival counter: barrier k of a launch is
// passed once the counter reaches k x (blocks), so the last block to arrive
// releases the others by its arrival alone. A block arrives with one
// acquire-release add (thread 0, after the block barrier: it publishes the
// block's writes of the phase) and polls the counter with acquire loads
// (the adds form one release sequence, so reading the final count acquires
// every block's writes). Every data read across blocks goes through L2
// (ld.global.cg), ordered after the acquire by the block barrier. The count
// wraps modulo 2^32; the comparison is of the signed difference.
__device__ __forceinline__ void gbar(const Grp &g)
{
    Scal *gs = g.gs;
    __syncthreads();
    if (tid_of() == 0) {
        const unsigned k = *g.gen + 1u;
        const unsigned target = k * (unsigned)g.nb;
        unsigned long long *tr =
            (g.trace && k <= (unsigned)g.trace_bars) ? g.trace + 2 * ((size_t)k * g.nb + g.rank) : nullptr;
        if (tr) tr[0] = globaltimer();
        unsigned c = atom_add_acq_rel(&gs->bar_count, 1u) + 1u;
        unsigned long long spins = 0;
        while ((int)(c - target) < 0) {
            if (spins++ >= g.spin_limit) {
                atomicCAS(&gs->status, 0, GEA_ERR_TIMEOUT);
                break;
            }
            c = ld_acquire(&gs->bar_count);
        }
        if (tr) tr[1] = globaltimer();
        *g.gen = k;
        s_stop = rdi(&gs->status) != 0 || s_ctl.status != 0;
    }
    __syncthreads();
}

// Every block leaves through here (all threads): the last of the launch's
// blocks to leave sets the arrival counter back to zero for the next launch
// (no block of this launch arrives again).
__device__ __forceinline__ void leave(const Grp &g)
{
    __syncthreads();
    if (tid_of() == 0 && atom_add_acq_rel(&g.gs->bar_exit, 1u) == (unsigned)g.nb - 1u) {
        g.gs->bar_count = 0u;
        g.gs->bar_exit = 0u;
    }
}

// Barrier with a deterministic grid-wide sum of NV per-thread values, which
// every block completes: it adds the block partials in a fixed order and
// thread 0 runs fin(tot) on the block's copy of the scalars. T is the type
// of the per-thread values and of the block sums (FP32 for the inner solves
// of the mixed-precision step); block partials and the total are FP64. The
// partials alternate between two buffers by barrier parity: a block
// writes a buffer again only two barriers later, after every block has read
// it.
template <int NV, class T, class Fin>
__device__ __forceinline__ void rbar(const Grp &g, const T (&v)[NV], double *red, double *partials, Fin fin)
{
    static_assert(NV <= kRedVals, "the block-sum scratch holds kRedVals values per thread");
    const int tid = tid_of();
    const int nb = g.nb;
    double *pb = partials + kGcntDoubles + (size_t)(*g.gen & 1u) * kRedVals * nb;
    T bt[NV];
    block_sum<NV, T>(v, reinterpret_cast<T *>(red), bt);
    if (tid == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) pb[(size_t)j * nb + g.rank] = (double)bt[j];
    }
    gbar(g);
    double s[NV], tot[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        s[j] = 0.0;
        for (int b = tid; b < nb; b += NTHREADS) s[j] += __ldcg(&pb[(size_t)j * nb + b]);
    }
    block_sum<NV>(s, red, tot);
    if (tid == 0) {
        fin(tot);
        if (s_ctl.status) {
            s_stop = 1;
            if (g.rank == 0) atomicCAS(&g.gs->status, 0, s_ctl.status);
        }
    }
    __syncthreads();
}

template <class F>
__device__ __forceinline__ void for_tiles(const Grp &g, const Geom &G, F f)
{
    const int tx = (G.nx + BX - 1) / BX, tz = (G.nz + BZ - 1) / BZ;
    const int nt = tx * tz;
    for (int t = g.rank; t < nt; t += g.nb) f(t % tx, t / tx);
}

__device__ __forceinline__ bool stop(const Scal *) { return s_stop != 0; }

// End of a step: its counters into the block's copy and, from block rank 0,
// into the context (what the host reads).
__device__ __forceinline__ void end_step(const Grp &g)
{
    gbar(g);
    if (tid_of() == 0 && !s_stop) {
        Scal &c = s_ctl;
        c.steps_done += 1;
        c.last_sweeps[0] = c.sweeps[0];
        c.last_sweeps[1] = c.sweeps[1];
        for (int k = 0; k < 4; ++k) {
            c.last_cg_iters[k] = c.cg_iters[k];
            c.last_cg_relres[k] = c.cg_relres[k];
        }
        c.last_status = 0;
        if (g.rank == 0) {
            Scal *gs = g.gs;
            gs->steps_done = c.steps_done;
            gs->last_sweeps[0] = c.last_sweeps[0];
            gs->last_sweeps[1] = c.last_sweeps[1];
            for (int k = 0; k < 4; ++k) {
                gs->last_cg_iters[k] = c.last_cg_iters[k];
                gs->last_cg_relres[k] = c.last_cg_relres[k];
            }
            gs->last_status = 0;
            gs->press_ns = c.press_ns;
        }
    }
}

// One time step reading a.S and writing a.N. Returns false if the step did
// not complete (a device error is set).
__device__ bool run_step(const PersistArgs &P, const StepArgs &a, const Grp &g, double *sm, double *red)
{
    Scal *sc = &s_ctl;   // the block's copy (decisions); g.gs holds the published values
    const Geom &G = a.G;
    const Level *L = P.L;
    const int nlev = P.nlev;

    // ---- Smagorinsky eddy viscosity of the step (LES) ----
    if (a.F.les) {
        for_tiles(g, G, [&](int bx, int bz) { ph_les(a, sm, bx, bz); });
        gbar(g);
        if (stop(sc)) return false;
    }
    // ---- Step 1: continuity predictor, transport operator, momentum RHS,
    // and the first Jacobi sweep of the momentum predictor (from u^n, which
    // needs no barrier) into ua, wa ----
    {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for_tiles(g, G, [&](int bx, int bz) { ph_pred_sweep(a, sm, bx, bz, acc); });
        rbar<4>(g, acc, red, a.partials, [&](const double (&t)[4]) {
            const double tb[2] = {t[0], t[1]}, tr[2] = {t[2], t[3]};
            fin_pred(sc, tb);
            for (int c = 0; c < 4; ++c) { sc->cg_iters[c] = 0; sc->cg_relres[c] = 0.0; }
            sc->sweeps[1] = 0;
            sc->press_ns = 0ull;
            fin_mom(sc, tr, a.jac_rtol2);
            if (!sc->done[LOOP_MOM] && !sc->status && sc->sweeps[0] >= P.jac_maxit) sc->status = GEA_ERR_NOCONV;
        });
    }
    if (stop(sc)) return false;
    // implicit momentum predictor: Jacobi until the sweep whose residual met
    // the tolerance
    const double *uin = a.ua, *win = a.wa;
    double *uout = a.ub, *wout = a.wb;
    while (!sc->done[LOOP_MOM]) {
        double acc[2] = {0.0, 0.0};
        for_tiles(g, G, [&](int bx, int bz) { ph_mom(a, uin, win, uout, wout, sm, bx, bz, acc); });
        rbar<2>(g, acc, red, a.partials, [&](const double (&t)[2]) {
            fin_mom(sc, t, a.jac_rtol2);
            if (!sc->done[LOOP_MOM] && !sc->status && sc->sweeps[0] >= P.jac_maxit) sc->status = GEA_ERR_NOCONV;
        });
        const double *tu = uin, *tw = win;
        uin = uout; win = wout;
        uout = const_cast<double *>(tu); wout = const_cast<double *>(tw);
        if (stop(sc)) break;
    }
    if (stop(sc)) return false;
    const double *u1 = uin, *w1 = win;

    // ---- Step 2: enthalpy right-hand side with the first enthalpy sweep
    // (from h^n) into ha, then temperature, rho^{n+2/3} ----
    {
        double acc[2] = {0.0, 0.0};
        for_tiles(g, G, [&](int bx, int bz) { ph_enth_rhs_sweep(a, u1, w1, a.ha, sm, bx, bz, acc); });
        rbar<2>(g, acc, red, a.partials, [&](const double (&t)[2]) {
            const double tb[1] = {t[0]}, tr[1] = {t[1]};
            fin_enth_rhs(sc, tb);
            fin_enth(sc, tr, a.jac_rtol2);
            if (!sc->done[LOOP_ENTH] && !sc->status && sc->sweeps[1] >= P.jac_maxit) sc->status = GEA_ERR_NOCONV;
        });
    }
    if (stop(sc)) return false;
    const double *hin = a.ha;
    double *hout = a.hb;
    while (!sc->done[LOOP_ENTH]) {
        double acc[1] = {0.0};
        for_tiles(g, G, [&](int bx, int bz) { ph_enth(a, hin, hout, sm, bx, bz, acc); });
        rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) {
            fin_enth(sc, t, a.jac_rtol2);
            if (!sc->done[LOOP_ENTH] && !sc->status && sc->sweeps[1] >= P.jac_maxit) sc->status = GEA_ERR_NOCONV;
        });
        const double *t = hin;
        hin = hout;
        hout = const_cast<double *>(t);
        if (stop(sc)) break;
    }
    if (stop(sc)) return false;
    const double *h1 = hin;
    // the EOS update, and H(u^{n+1/3}) of the first corrector, which reads
    // nothing the EOS phase writes
    for_tiles(g, G, [&](int bx, int bz) { ph_eos(a, L[0], h1, sm, bx, bz); });
    for_tiles(g, G, [&](int bx, int bz) { ph_H(a, u1, w1, sm, bx, bz); });
    gbar(g);
    for (int l = 0; l + 1 < nlev; ++l) {
        for_tiles(g, L[l + 1].G, [&](int bx, int bz) { ph_coarsen(L[l], L[l + 1], a.F.omega, bx, bz); });
        gbar(g);
    }
    if (stop(sc)) return false;
    if (g.rank == 0 && tid_of() == 0) {
        g.gs->u1_slot = (u1 == a.ub);
        g.gs->h1_slot = (h1 == a.hb);
    }

    // ---- Step 3: PISO correctors ----
    for (int c = 0; c < P.n_corr; ++c) {
        if (c > 0) {
            for_tiles(g, G, [&](int bx, int bz) { ph_H(a, a.N.u, a.N.w, sm, bx, bz); });
            gbar(g);
        }
        unsigned long long t0 = 0;
        if (g.rank == 0 && tid_of() == 0) t0 = globaltimer();
        {
            double acc[2] = {0.0, 0.0};
            const double *xin = c == 0 ? a.S.pp : a.N.pp;
            for_tiles(g, G, [&](int bx, int bz) { ph_helm_rhs(a, L[0], xin, a.N.pp, sm, bx, bz, acc); });
            rbar<2>(g, acc, red, a.partials, [&](const double (&t)[2]) { fin_helm(sc, t, a.cg_rtol2, c); });
        }
        // z = M^-1 r_0 (one V(1,1)-cycle), then the iterations
        auto vcycle_levels = [&](int lfirst) {
            for (int l = lfirst; l + 1 < nlev; ++l) {
                for_tiles(g, L[l].G, [&](int bx, int bz) { ph_mg_down(L[l], L[l + 1], a.F.omega, sm, bx, bz); });
                gbar(g);
            }
            const Level &C = L[nlev - 1];
            for (int s = 0; s < P.ncoarse; ++s) {
                double *out = ((P.ncoarse - 1 - s) % 2 == 0) ? C.e2 : C.e;
                const double *in = (out == C.e2) ? C.e : C.e2;
                for_tiles(g, C.G, [&](int bx, int bz) { ph_mg_coarse(C, in, out, s == 0, sm, bx, bz); });
                gbar(g);
            }
            const double *res0 = res_of(L[0], sc->cg_it);
            for (int l = nlev - 2; l >= 0; --l) {
                double acc[1] = {0.0};
                const double *res = l == 0 ? res0 : L[l].r;
                for_tiles(g, L[l].G, [&](int bx, int bz) {
                    ph_mg_up(L[l], res, L[l + 1].e2, L[l + 1].G.P, L[l].e2, sm, bx, bz, acc);
                });
                if (l > 0) gbar(g);
                else rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) { fin_rz(sc, t); });
            }
        };
        if (!stop(sc) && !sc->done[LOOP_CG]) {
            if (nlev == 1) {
                double acc[1] = {0.0};
                for_tiles(g, G, [&](int bx, int bz) { ph_mg_single(L[0], L[0].e2, sm, bx, bz, acc); });
                rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) { fin_rz(sc, t); });
            } else {
                vcycle_levels(0);
            }
        }
        while (!stop(sc) && !sc->done[LOOP_CG]) {
            // p = z + beta p, q = A p
            const int it = sc->cg_it;
            const double *pold = (it & 1) ? a.p1 : a.p0;
            double *pnew = (it & 1) ? a.p0 : a.p1;
            {
                const double beta = sc->beta;
                double acc[1] = {0.0};
                for_tiles(g, G, [&](int bx, int bz) { ph_pspmv<double>(L[0], pold, pnew, a.q, beta, sm, bx, bz, acc); });
                rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) { fin_pq(sc, t); });
            }
            // x += alpha p, r -= alpha q, with the first step of the next V-cycle
            const double alpha = sc->alpha;
            auto cap = [&] {
                if (!sc->done[LOOP_CG] && !sc->status && sc->cg_it >= P.cg_maxit) sc->status = GEA_ERR_NOCONV;
            };
            if (nlev == 1) {
                double acc[2] = {0.0, 0.0};
                for_tiles(g, G, [&](int bx, int bz) {
                    ph_update_single<double>(L[0], a.q, res_of(L[0], it), res_of(L[0], it + 1), a.N.pp,
                                             pnew, alpha, sm, bx, bz, acc);
                });
                rbar<2>(g, acc, red, a.partials, [&](const double (&t)[2]) {
                    const double t0[1] = {t[0]}, t1[1] = {t[1]};
                    fin_update(sc, t0, a.cg_rtol2);
                    fin_rz(sc, t1);
                    cap();
                });
            } else {
                double acc[1] = {0.0};
                for_tiles(g, G, [&](int bx, int bz) {
                    ph_update_down<double>(L[0], L[1], a.q, res_of(L[0], it), res_of(L[0], it + 1), a.N.pp,
                                           pnew, alpha, a.F.omega, sm, bx, bz, acc);
                });
                rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) {
                    fin_update(sc, t, a.cg_rtol2);
                    cap();
                });
                if (!stop(sc) && !sc->done[LOOP_CG]) vcycle_levels(1);
            }
        }
        if (stop(sc)) return false;
        if (g.rank == 0 && tid_of() == 0) sc->press_ns += globaltimer() - t0;
        for_tiles(g, G, [&](int bx, int bz) { ph_correct(a, sm, bx, bz); });
        if (c + 1 < P.n_corr) gbar(g);
    }
    end_step(g);
    return !stop(sc);
}

// One mixed-precision time step (the phases of the graph's mixed step, in
// its order): FP64 residuals, FP32 Jacobi and MG-CG solves of the
// increments, FP64 updates. Returns false if the step did not complete.
__device__ bool run_step_mixed(const PersistArgs &P, const MixedPersist &X, const StepArgs &a, const Grp &g,
                               double *sm, double *red)
{
    Scal *sc = &s_ctl;   // the block's copy (decisions); g.gs holds the published values
    const Geom &G = a.G;
    const MixedArgs &m = X.m;
    const LevelF *L = X.Lf;
    const int nlev = X.nlev;
    const Level &L0 = P.L[0];
    if (g.rank == 0 && tid_of() == 0) g.gs->u1_slot = g.gs->h1_slot = 0;

    if (a.F.les) {
        for_tiles(g, G, [&](int bx, int bz) { ph_les(a, sm, bx, bz); });
        gbar(g);
        if (stop(sc)) return false;
    }
    // ---- Step 1: FP64 residuals r0 = b - T(u^n), FP32 operator, first FP32
    // sweep from zero ----
    {
        double acc[2] = {0.0, 0.0};
        for_tiles(g, G, [&](int bx, int bz) { ph_pred_t<true>(a, m, sm, bx, bz, acc); });
        rbar<2>(g, acc, red, a.partials, [&](const double (&t)[2]) {
            fin_pred(sc, t);
            for (int c = 0; c < 4; ++c) { sc->cg_iters[c] = 0; sc->cg_relres[c] = 0.0; }
            sc->sweeps[1] = 0;
            sc->press_ns = 0ull;
        });
    }
    if (stop(sc)) return false;
    const float *ui = m.du[0], *wi = m.dw[0];
    float *uo = m.du[1], *wo = m.dw[1];
    for (;;) {
        float acc[2] = {0.0f, 0.0f};
        for_tiles(g, G, [&](int bx, int bz) {
            ph_sweep2<float, BC_U, BC_W>(G, a.F, m.T, m.dinvu, m.r0u, m.r0w, ui, wi, uo, wo, sm, bx, bz, acc);
        });
        rbar<2>(g, acc, red, a.partials, [&](const double (&t)[2]) {
            fin_mom(sc, t, m.tol2);
            if (!sc->done[LOOP_MOM] && !sc->status && sc->sweeps[0] >= P.jac_maxit) sc->status = GEA_ERR_NOCONV;
        });
        const float *tu = ui, *tw = wi;
        ui = uo; wi = wo;
        uo = const_cast<float *>(tu); wo = const_cast<float *>(tw);
        if (stop(sc) || sc->done[LOOP_MOM]) break;
    }
    if (stop(sc)) return false;

    // ---- Step 2: u^{n+1/3} = u^n + du, the enthalpy residual at h^n and the
    // first FP32 sweep; FP32 Jacobi on dh ----
    {
        MixedArgs mm = m;   // the momentum increments end in the buffers ui, wi
        mm.du[0] = const_cast<float *>(ui);
        mm.dw[0] = const_cast<float *>(wi);
        double acc[1] = {0.0};
        for_tiles(g, G, [&](int bx, int bz) {
            ph_enth_rhs_t<true>(a, mm, nullptr, nullptr, nullptr, sm, bx, bz, acc);
        });
        rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) { fin_enth_rhs(sc, t); });
    }
    if (stop(sc)) return false;
    const float *hi = m.dh[0];
    float *ho = m.dh[1];
    const float lc = (float)(a.F.mu - a.F.nuh);
    for (;;) {
        float acc[1] = {0.0f};
        for_tiles(g, G, [&](int bx, int bz) {
            ph_sweep1<float, BC_EVEN>(G, a.F, m.T, m.dinvh, m.r0h, lc, hi, ho, sm, bx, bz, acc);
        });
        rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) {
            fin_enth(sc, t, m.tol2);
            if (!sc->done[LOOP_ENTH] && !sc->status && sc->sweeps[1] >= P.jac_maxit) sc->status = GEA_ERR_NOCONV;
        });
        const float *t = hi;
        hi = ho;
        ho = const_cast<float *>(t);
        if (stop(sc) || sc->done[LOOP_ENTH]) break;
    }
    if (stop(sc)) return false;
    // h^{n+1} = h^n + dh, the EOS update, the FP64 finest Helmholtz level and
    // its FP32 copy; H(u^{n+1/3}) of the first corrector reads nothing of it
    for_tiles(g, G, [&](int bx, int bz) { ph_eos_t<true>(a, L0, L[0], nullptr, hi, sm, bx, bz); });
    for_tiles(g, G, [&](int bx, int bz) { ph_H(a, a.ua, a.wa, sm, bx, bz); });
    gbar(g);
    for (int l = 0; l + 1 < nlev; ++l) {
        for_tiles(g, L[l + 1].G, [&](int bx, int bz) { ph_coarsen<float>(L[l], L[l + 1], a.F.omega, bx, bz); });
        gbar(g);
    }
    if (stop(sc)) return false;

    // ---- Step 3: PISO correctors, each pressure solve one defect correction ----
    for (int c = 0; c < P.n_corr; ++c) {
        if (c > 0) {
            for_tiles(g, G, [&](int bx, int bz) { ph_H(a, a.N.u, a.N.w, sm, bx, bz); });
            gbar(g);
        }
        unsigned long long t0 = 0;
        if (g.rank == 0 && tid_of() == 0) t0 = globaltimer();
        {
            double acc[2] = {0.0, 0.0};
            const double *xin = c == 0 ? a.S.pp : a.N.pp;
            for_tiles(g, G, [&](int bx, int bz) {
                ph_helm_rhs_t<true>(a, L0, L[0], m, xin, a.N.pp, sm, bx, bz, acc);
            });
            rbar<2>(g, acc, red, a.partials, [&](const double (&t)[2]) {
                fin_helm_mixed(sc, t, a.cg_rtol2, c);
            });
        }
        auto vcycle_levels = [&](int lfirst) {
            for (int l = lfirst; l + 1 < nlev; ++l) {
                for_tiles(g, L[l].G, [&](int bx, int bz) {
                    ph_mg_down<float>(L[l], L[l + 1], a.F.omega, sm, bx, bz);
                });
                gbar(g);
            }
            const LevelF &C = L[nlev - 1];
            for (int s = 0; s < P.ncoarse; ++s) {
                float *out = ((P.ncoarse - 1 - s) % 2 == 0) ? C.e2 : C.e;
                const float *in = (out == C.e2) ? C.e : C.e2;
                for_tiles(g, C.G, [&](int bx, int bz) { ph_mg_coarse<float>(C, in, out, s == 0, sm, bx, bz); });
                gbar(g);
            }
            const float *res0 = res_of(L[0], sc->cg_it);
            for (int l = nlev - 2; l >= 0; --l) {
                float acc[1] = {0.0f};
                const float *res = l == 0 ? res0 : L[l].r;
                for_tiles(g, L[l].G, [&](int bx, int bz) {
                    ph_mg_up<float>(L[l], res, L[l + 1].e2, L[l + 1].G.P, L[l].e2, sm, bx, bz, acc);
                });
                if (l > 0) gbar(g);
                else rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) { fin_rz(sc, t); });
            }
        };
        if (!stop(sc) && !sc->done[LOOP_CG]) {
            if (nlev == 1) {
                float acc[1] = {0.0f};
                for_tiles(g, G, [&](int bx, int bz) { ph_mg_single<float>(L[0], L[0].e2, sm, bx, bz, acc); });
                rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) { fin_rz(sc, t); });
            } else {
                vcycle_levels(0);
            }
        }
        while (!stop(sc) && !sc->done[LOOP_CG]) {
            const int it = sc->cg_it;
            const float *pold = (it & 1) ? m.p1 : m.p0;
            float *pnew = (it & 1) ? m.p0 : m.p1;
            {
                const double beta = sc->beta;
                float acc[1] = {0.0f};
                for_tiles(g, G, [&](int bx, int bz) {
                    ph_pspmv<float>(L[0], pold, pnew, m.q, beta, sm, bx, bz, acc);
                });
                rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) { fin_pq(sc, t); });
            }
            const double alpha = sc->alpha;
            auto cap = [&] {
                if (!sc->done[LOOP_CG] && !sc->status && sc->cg_it >= P.cg_maxit) sc->status = GEA_ERR_NOCONV;
            };
            if (nlev == 1) {
                float acc[2] = {0.0f, 0.0f};
                for_tiles(g, G, [&](int bx, int bz) {
                    ph_update_single<float>(L[0], m.q, res_of(L[0], it), res_of(L[0], it + 1), m.x, pnew, alpha,
                                            sm, bx, bz, acc);
                });
                rbar<2>(g, acc, red, a.partials, [&](const double (&t)[2]) {
                    const double t0[1] = {t[0]}, t1[1] = {t[1]};
                    fin_update(sc, t0, m.tol2);
                    fin_rz(sc, t1);
                    cap();
                });
            } else {
                float acc[1] = {0.0f};
                for_tiles(g, G, [&](int bx, int bz) {
                    ph_update_down<float>(L[0], L[1], m.q, res_of(L[0], it), res_of(L[0], it + 1), m.x, pnew,
                                          alpha, a.F.omega, sm, bx, bz, acc);
                });
                rbar<1>(g, acc, red, a.partials, [&](const double (&t)[1]) {
                    fin_update(sc, t, m.tol2);
                    cap();
                });
                if (!stop(sc) && !sc->done[LOOP_CG]) vcycle_levels(1);
            }
        }
        if (stop(sc)) return false;
        // p' += dp, then the FP64 correction
        for_tiles(g, G, [&](int bx, int bz) { ph_p_apply(a, m, bx, bz); });
        gbar(g);
        if (g.rank == 0 && tid_of() == 0) sc->press_ns += globaltimer() - t0;
        for_tiles(g, G, [&](int bx, int bz) { ph_correct(a, sm, bx, bz); });
        if (c + 1 < P.n_corr) gbar(g);
    }
    end_step(g);
    return !stop(sc);
}

__global__ void __launch_bounds__(NTHREADS, 3) k_persistent(PersistArgs P)
{
    extern __shared__ double dsm[];
    double *sm = dsm;
    double *red = dsm + kTileSmem;
    // an error status is sticky until the next set_state, which clears it
    __shared__ unsigned gen;
    Scal *gs = P.a[0].sc;
    if (tid_of() == 0) {
        s_stop = rdi(&gs->status) != 0;
        gen = 0u;
    }
    load_ctl(gs);
    __syncthreads();
    const Grp g{(int)blockIdx.x, (int)gridDim.x, &gen, gs, P.spin_limit, P.a[0].trace, P.a[0].trace_bars};
    trace_entry(g);
    if (!s_stop) {
        if (blockIdx.x == 0 && tid_of() == 0) gs->launches += 1;
        for (int s = 0; s < P.nsteps; ++s) {
            const int slot = (P.first_slot + s) & 1;
            if (!run_step(P, P.a[slot], g, sm, red)) break;
        }
        if (blockIdx.x == 0 && tid_of() == 0 && rdi(&gs->status)) gs->last_status = rdi(&gs->status);
    }
    leave(g);
}

constexpr size_t kPersistSmem = (size_t)(kTileSmem + kRedVals * NTHREADS) * sizeof(double);

// The mixed-precision step as one cooperative launch (small grids).
__global__ void __launch_bounds__(NTHREADS, 3) k_persistent_mixed(PersistArgs P, MixedPersist X)
{
    extern __shared__ double dsm[];
    double *sm = dsm;
    double *red = dsm + kTileSmem;
    __shared__ unsigned gen;
    Scal *gs = P.a[0].sc;
    if (tid_of() == 0) {
        s_stop = rdi(&gs->status) != 0;
        gen = 0u;
    }
    load_ctl(gs);
    __syncthreads();
    const Grp g{(int)blockIdx.x, (int)gridDim.x, &gen, gs, P.spin_limit, P.a[0].trace, P.a[0].trace_bars};
    trace_entry(g);
    if (!s_stop) {
        if (blockIdx.x == 0 && tid_of() == 0) gs->launches += 1;
        for (int s = 0; s < P.nsteps; ++s) {
            const int slot = (P.first_slot + s) & 1;
            if (!run_step_mixed(P, X, P.a[slot], g, sm, red)) break;
        }
        if (blockIdx.x == 0 && tid_of() == 0 && rdi(&gs->status)) gs->last_status = rdi(&gs->status);
    }
    leave(g);
}

// An ensemble of independent contexts in one cooperative launch. The blocks
// form groups (table `groups`: ngroups + 1 first blocks, ngroups + 1 first
// entries of the member list, then the member list): a group of several
// blocks runs one member, with its own barrier and reductions over those
// blocks only, so members whose solves take different iteration counts never
// wait for one another; a group of one block may run several small members,
// one after another, each as a one-block grid. Each block keeps the argument
// block of the member it runs in shared memory: a PersistArgs block of
// `stride` bytes per member, for the mixed-precision step (MX) followed by
// the member's MixedPersist.
template <bool MX>
__global__ void __launch_bounds__(NTHREADS, 3) k_ensemble(const char *Pm, int stride, const int *groups, int ngroups)
{
    extern __shared__ double dsm[];
    double *sm = dsm;
    double *red = dsm + kTileSmem;
    PersistArgs *Ps = reinterpret_cast<PersistArgs *>(dsm + kTileSmem + kRedVals * NTHREADS);
    const int tid = tid_of();
    const int *gb = groups, *gm = groups + ngroups + 1, *order = gm + ngroups + 1;
    int lo = 0, hi = ngroups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (__ldg(&gb[mid]) <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const int b0 = __ldg(&gb[lo]), nbk = __ldg(&gb[lo + 1]) - b0;
    const int i1 = __ldg(&gm[lo + 1]);
    __shared__ unsigned gen;
    for (int i = __ldg(&gm[lo]); i < i1; ++i) {
        const int m = __ldg(&order[i]);
        __syncthreads();   // nothing reads the previous member's arguments any more
        {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(Pm + (size_t)m * stride);
            uint32_t *dst = reinterpret_cast<uint32_t *>(Ps);
            for (int w = tid; w < stride / 4; w += NTHREADS) dst[w] = __ldg(&src[w]);
        }
        __syncthreads();
        const PersistArgs &P = *Ps;
        const MixedPersist &X = *reinterpret_cast<const MixedPersist *>(reinterpret_cast<const char *>(Ps) +
                                                                        sizeof(PersistArgs));
        Scal *sc = P.a[0].sc;
        if (tid == 0) {
            s_stop = rdi(&sc->status) != 0;
            gen = 0u;
        }
        load_ctl(sc);
        __syncthreads();
        const Grp g{(int)blockIdx.x - b0, nbk, &gen, sc, P.spin_limit, nullptr, 0};
        if (!s_stop) {
            if (g.rank == 0 && tid == 0) sc->launches += 1;
            for (int s = 0; s < P.nsteps; ++s) {
                const int slot = (P.first_slot + s) & 1;
                const bool ok =
                    MX ? run_step_mixed(P, X, P.a[slot], g, sm, red) : run_step(P, P.a[slot], g, sm, red);
                if (!ok) break;
            }
            if (g.rank == 0 && tid == 0 && rdi(&sc->status)) sc->last_status = rdi(&sc->status);
        }
        leave(g);
    }
}

// bytes of one member's argument block and the ensemble kernels' shared memory
constexpr size_t kArgsFp64 = sizeof(PersistArgs);
constexpr size_t kArgsMixed = sizeof(PersistArgs) + sizeof(MixedPersist);
constexpr size_t kEnsembleSmem = kPersistSmem + (kArgsFp64 + 15) / 16 * 16;
constexpr size_t kEnsembleSmemMixed = kPersistSmem + (kArgsMixed + 15) / 16 * 16;

int ensemble_max_blocks(int mixed)
{
    int dev = 0, sms = 0, per_sm = 0;
    const void *k = mixed ? (const void *)k_ensemble<true> : (const void *)k_ensemble<false>;
    const size_t smem = mixed ? kEnsembleSmemMixed : kEnsembleSmem;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NTHREADS, smem) != cudaSuccess) return 0;
    return per_sm * sms;
}

cudaError_t launch_ensemble(const void *Pm, int mixed, const int *groups, int ngroups, int blocks, cudaStream_t st)
{
    const char *P = static_cast<const char *>(Pm);
    int stride = (int)(mixed ? kArgsMixed : kArgsFp64);
    void *args[] = {&P, &stride, &groups, &ngroups};
    const void *k = mixed ? (const void *)k_ensemble<true> : (const void *)k_ensemble<false>;
    return cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(BX, BZ), args,
                                       mixed ? kEnsembleSmemMixed : kEnsembleSmem, st);
}

int persistent_max_blocks()
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPersistSmem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent, NTHREADS, kPersistSmem) !=
        cudaSuccess)
        return 0;
    return per_sm * sms;
}

cudaError_t launch_persistent(const StepArgs a[2], const Level *L, int nlev, int ncoarse, int n_corr,
                              int jac_maxit, int cg_maxit, int first_slot, int nsteps, int blocks,
                              long long wait_polls, cudaStream_t st)
{
    if (nlev < 1 || nlev > kMaxLevels) return cudaErrorInvalidValue;
    PersistArgs P;
    memset(&P, 0, sizeof(P));
    P.a[0] = a[0];
    P.a[1] = a[1];
    for (int l = 0; l < nlev; ++l) P.L[l] = L[l];
    P.nlev = nlev;
    P.ncoarse = ncoarse;
    P.nsteps = nsteps;
    P.first_slot = first_slot;
    P.n_corr = n_corr;
    P.jac_maxit = jac_maxit;
    P.cg_maxit = cg_maxit;
    P.spin_limit = spin_limit_of(wait_polls);
    void *args[] = {&P};
    return cudaLaunchCooperativeKernel((const void *)k_persistent, dim3(blocks), dim3(BX, BZ), args,
                                       kPersistSmem, st);
}

int persistent_mixed_max_blocks()
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k_persistent_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPersistSmem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent_mixed, NTHREADS, kPersistSmem) !=
        cudaSuccess)
        return 0;
    return per_sm * sms;
}

cudaError_t launch_persistent_mixed(const StepArgs a[2], const Level &L0, const MixedArgs &m, const LevelF *Lf,
                                    int nlev, int ncoarse, int n_corr, int jac_maxit, int cg_maxit,
                                    int first_slot, int nsteps, int blocks, long long wait_polls,
                                    cudaStream_t st)
{
    if (nlev < 1 || nlev > kMaxLevels) return cudaErrorInvalidValue;
    PersistArgs P;
    memset(&P, 0, sizeof(P));
    P.a[0] = a[0];
    P.a[1] = a[1];
    P.L[0] = L0;
    P.nlev = 1;
    P.ncoarse = ncoarse;
    P.nsteps = nsteps;
    P.first_slot = first_slot;
    P.n_corr = n_corr;
    P.jac_maxit = jac_maxit;
    P.cg_maxit = cg_maxit;
    P.spin_limit = spin_limit_of(wait_polls);
    MixedPersist X;
    memset(&X, 0, sizeof(X));
    X.m = m;
    for (int l = 0; l < nlev; ++l) X.Lf[l] = Lf[l];
    X.nlev = nlev;
    void *args[] = {&P, &X};
    return cudaLaunchCooperativeKernel((const void *)k_persistent_mixed, dim3(blocks), dim3(BX, BZ), args,
                                       kPersistSmem, st);
}

}  // namespace

// the host entry points of this tile shape (external linkage: the shape
// table in gea_persistent.cu refers to it)
extern const PersistOps ops;
const PersistOps ops = {BX,
                        BZ,
                        persistent_max_blocks,
                        persistent_mixed_max_blocks,
                        ensemble_max_blocks,
                        launch_persistent,
                        launch_persistent_mixed,
                        launch_ensemble};
