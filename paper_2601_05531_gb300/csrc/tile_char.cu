// tile_char.cu -- instantiates the tile kernel for MODE_CHAR.
#include "tile_dispatch.cuh"

namespace dnatok {
template cudaError_t launch_mode<MODE_CHAR>(int, const TileParams &, const LaunchShape &, cudaStream_t,
                                       int);
}  // namespace dnatok
