// tile_dispatch.cuh -- host-side launch templates of the tile kernel; each
// mode is instantiated in its own translation unit (tile_<mode>.cu) so the
// library builds in parallel.
#pragma once
#include "internal.h"
#include "tile_kernel.cuh"

namespace dnatok {

template <int MODE, int BSRC, int NT, int TILE, int NSUB>
static cudaError_t launch_one(const TileParams &p, cudaStream_t s, int sm_count, int ctas_per_sm) {
    constexpr int SMEM = tile_smem_bytes(TILE, NT);
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(tile_kernel<MODE, BSRC, NT, TILE, NSUB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    long long grid = (long long)sm_count * ctas_per_sm;
    if (grid > p.n_chunks) grid = p.n_chunks;
    if (grid < 1) grid = 1;
    if (!p.gate) {
        tile_kernel<MODE, BSRC, NT, TILE, NSUB><<<(unsigned)grid, NT, SMEM, s>>>(p);
        return cudaGetLastError();
    }
    // behind the direct path: launched as a programmatic dependent so its
    // launch overlaps the direct kernel's tail (it waits for it on the device)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tile_kernel<MODE, BSRC, NT, TILE, NSUB>, p);
}

// The supported shapes: tile bytes, threads, tiles per chunk.
#define DNATOK_SHAPES(X)        \
    X(8192, 256, 8)             \
    X(16384, 256, 4)            \
    X(16384, 256, 8)            \
    X(32768, 512, 4)

template <int MODE, int BSRC>
static cudaError_t launch_shape(const TileParams &p, const LaunchShape &sh, cudaStream_t s,
                                int sm_count) {
    const int c = sh.ctas_per_sm;
#define DNATOK_TRY(T, N, C)                                                   \
    if (sh.tile == T && sh.threads == N && sh.chunk_tiles == C)               \
        return launch_one<MODE, BSRC, N, T, C>(p, s, sm_count, c);
    DNATOK_SHAPES(DNATOK_TRY)
#undef DNATOK_TRY
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
