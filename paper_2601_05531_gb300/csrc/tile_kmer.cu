// tile_kmer.cu -- instantiates the tile kernel for MODE_KMER.
#include "tile_dispatch.cuh"

namespace dnatok {
template cudaError_t launch_mode<MODE_KMER>(int, const TileParams &, const LaunchShape &, cudaStream_t,
                                       int);
}  // namespace dnatok
