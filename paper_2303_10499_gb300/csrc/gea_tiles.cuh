// gea_tiles.cuh -- the tile phase functions (gea_tiles_body.cuh) for the
// 32 x 8 tile of the per-phase kernels, in namespace gea::tiles.
#pragma once

#include "gea_internal.cuh"

namespace gea {
namespace tiles {
constexpr bool kPrefetch = false;   // per-phase kernels: occupancy first
#include "gea_tiles_body.cuh"
}  // namespace tiles
}  // namespace gea
