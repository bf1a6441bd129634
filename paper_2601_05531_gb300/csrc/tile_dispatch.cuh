// tile_dispatch.cuh -- host-side launch templates of the tile kernel; each
// mode is instantiated in its own translation unit (tile_<mode>.cu) so the
// library builds in parallel.
#pragma once
#include "internal.h"
#include "tile_kernel.cuh"

namespace dnatok {

template <int MODE, int BSRC, int NT, int TILE>
static cudaError_t launch_one(const TileParams &p, cudaStream_t s, int sm_count, int ctas_per_sm) {
    constexpr int SMEM = tile_smem_bytes(TILE, NT);
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(tile_kernel<MODE, BSRC, NT, TILE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    long long grid = (long long)sm_count * ctas_per_sm;
    if (grid > p.n_tiles) grid = p.n_tiles;
    if (grid < 1) grid = 1;
    tile_kernel<MODE, BSRC, NT, TILE><<<(unsigned)grid, NT, SMEM, s>>>(p);
    return cudaGetLastError();
}

template <int MODE, int BSRC>
static cudaError_t launch_shape(const TileParams &p, const LaunchShape &sh, cudaStream_t s,
                                int sm_count) {
    const int c = sh.ctas_per_sm;
    if (sh.tile == 8192 && sh.threads == 256) return launch_one<MODE, BSRC, 256, 8192>(p, s, sm_count, c);
    if (sh.tile == 16384 && sh.threads == 256) return launch_one<MODE, BSRC, 256, 16384>(p, s, sm_count, c);
    if (sh.tile == 16384 && sh.threads == 512) return launch_one<MODE, BSRC, 512, 16384>(p, s, sm_count, c);
    if (sh.tile == 32768 && sh.threads == 512) return launch_one<MODE, BSRC, 512, 32768>(p, s, sm_count, c);
    return cudaErrorInvalidValue;
}

template <int MODE>
cudaError_t launch_mode(int bsrc, const TileParams &p, const LaunchShape &sh, cudaStream_t s,
                        int sm_count) {
    switch (bsrc) {
    case BSRC_LIST: return launch_shape<MODE, BSRC_LIST>(p, sh, s, sm_count);
    case BSRC_FASTA: return launch_shape<MODE, BSRC_FASTA>(p, sh, s, sm_count);
    case BSRC_FLAGS: return launch_shape<MODE, BSRC_FLAGS>(p, sh, s, sm_count);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dnatok
