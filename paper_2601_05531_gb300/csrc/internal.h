// internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "dnatok.h"

namespace dnatok {

struct TileParams;

struct LaunchShape {
    int tile;         // bytes per tile
    int threads;      // threads per CTA
    int ctas_per_sm;  // resident CTAs per SM the grid is sized for
    int chunk_tiles;  // tiles per chunk (the unit of the look-back)
};

// Shape of the direct k-mer kernel: 512-byte slots per warp step, warp
// steps in its ring, resident CTAs per SM (0 = as many as fit).
struct DirectShape {
    int slots;
    int ring;
    int ctas_per_sm;
};

bool tile_shape_supported(const LaunchShape &sh);
bool direct_shape_supported(const DirectShape &sh);
cudaError_t launch_tile_kernel(int mode, int bsrc, const TileParams &p, const LaunchShape &sh,
                               cudaStream_t s, int sm_count);
cudaError_t launch_empty_chunk(const TileParams &p, int list_source, cudaStream_t s);

}  // namespace dnatok
