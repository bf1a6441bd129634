// tile_sym.cu -- instantiates the tile kernel for MODE_SYM.
#include "tile_dispatch.cuh"

namespace dnatok {
template cudaError_t launch_mode<MODE_SYM>(int, const TileParams &, const LaunchShape &, cudaStream_t,
                                       int);
}  // namespace dnatok
