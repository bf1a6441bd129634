// internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/dnatok.h"

namespace dnatok {

struct TileParams;

struct LaunchShape {
    int tile;
    int threads;
    int ctas_per_sm;
};

bool tile_shape_supported(const LaunchShape &sh);
cudaError_t launch_tile_kernel(int mode, int bsrc, const TileParams &p, const LaunchShape &sh,
                               cudaStream_t s, int sm_count);
cudaError_t launch_plan_list(const long long *off, long long n_bnd, long long n_bytes, int head_pad,
                             int tile, long long n_tiles, int *tile_rec,
                             unsigned long long *counter, int *status, cudaStream_t s);
cudaError_t launch_empty_chunk(const TileParams &p, int list_source, cudaStream_t s);

}  // namespace dnatok
