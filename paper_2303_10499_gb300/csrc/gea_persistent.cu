// gea_persistent.cu -- the persistent step kernels for the 32 x 8 tile (the
// default shape, also the tile of the per-phase kernels), the tile-shape
// table, and the argument blocks of ensemble launches.
#include "gea_internal.cuh"

#include <string.h>

namespace gea {
namespace tiles_32x8 {
constexpr int BX = 32;   // cells (threads) per tile row
constexpr int BZ = 8;    // rows per tile
constexpr bool kPrefetch = true;   // cell inputs loaded ahead of the tile barrier
#include "gea_tiles_body.cuh"
#include "gea_persistent_body.cuh"
}  // namespace tiles_32x8

namespace tiles_16x16 {
extern const PersistOps ops;
}
namespace tiles_64x4 {
extern const PersistOps ops;
}

const PersistOps &persist_ops(int shape)
{
    switch (shape) {
    case SHAPE_16x16: return tiles_16x16::ops;
    case SHAPE_64x4: return tiles_64x4::ops;
    default: return tiles_32x8::ops;
    }
}

size_t persist_args_bytes(int mixed) { return mixed ? sizeof(PersistArgs) + sizeof(MixedPersist) : sizeof(PersistArgs); }

void persist_args_fill_mixed(void *dst, const StepArgs a[2], const Level &L0, const MixedArgs &m,
                             const LevelF *Lf, int nlev, int ncoarse, int n_corr, int jac_maxit, int cg_maxit,
                             int first_slot, int nsteps, long long wait_polls)
{
    persist_args_fill(dst, a, &L0, 1, ncoarse, n_corr, jac_maxit, cg_maxit, first_slot, nsteps, wait_polls);
    MixedPersist X;
    memset(&X, 0, sizeof(X));
    X.m = m;
    for (int l = 0; l < nlev && l < kMaxLevels; ++l) X.Lf[l] = Lf[l];
    X.nlev = nlev;
    memcpy(static_cast<char *>(dst) + sizeof(PersistArgs), &X, sizeof(X));
}

void persist_args_fill(void *dst, const StepArgs a[2], const Level *L, int nlev, int ncoarse, int n_corr,
                       int jac_maxit, int cg_maxit, int first_slot, int nsteps, long long wait_polls)
{
    PersistArgs P;
    memset(&P, 0, sizeof(P));
    P.a[0] = a[0];
    P.a[1] = a[1];
    for (int l = 0; l < nlev && l < kMaxLevels; ++l) P.L[l] = L[l];
    P.nlev = nlev;
    P.ncoarse = ncoarse;
    P.nsteps = nsteps;
    P.first_slot = first_slot;
    P.n_corr = n_corr;
    P.jac_maxit = jac_maxit;
    P.cg_maxit = cg_maxit;
    P.spin_limit = spin_limit_of(wait_polls);
    memcpy(dst, &P, sizeof(P));
}

}  // namespace gea
