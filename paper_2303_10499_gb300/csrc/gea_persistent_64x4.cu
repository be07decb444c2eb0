// gea_persistent_64x4.cu -- the persistent step kernels (FP64, mixed
// precision, ensemble) for the 64 x 4 tile, one of the shapes the
// tile-shape autotuner chooses from (gea_set_tile_shape).
#include "gea_internal.cuh"

#include <string.h>

namespace gea {
namespace tiles_64x4 {
constexpr int BX = 64;   // cells (threads) per tile row
constexpr int BZ = 4;   // rows per tile
constexpr bool kPrefetch = true;   // cell inputs loaded ahead of the tile barrier
#include "gea_tiles_body.cuh"
#include "gea_persistent_body.cuh"
}  // namespace tiles_64x4
}  // namespace gea
