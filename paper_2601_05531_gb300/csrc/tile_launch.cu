// tile_launch.cu -- dispatch of the tile kernel and the zero-byte chunk
// kernel, with their host-side launchers.
#include "internal.h"
#include "tile_kernel.cuh"

namespace dnatok {

// A chunk with no bytes: only boundaries (all at one position).  Closes the
// open record (emitting its UNK tail in k-mer mode) and writes the offsets.
__global__ void empty_chunk_kernel(TileParams p, int list_source) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (dev_failed(p.status)) return;
    const int k = p.k;
    const KDiv kd = make_kdiv(k);
    const Agg c = p.carry_in ? p.carry_in->a : agg_identity();
    const long long nbz = list_source ? p.n_bnd : (long long)p.end_boundary;
    Agg z = agg_identity();
    z.nb = nbz;
    const Agg incl = agg_combine(c, z, kd);
    if (nbz > 0) {
        long long tclose = 0;
        if (c.nb > 0) {
            tclose = c.d - kd.div(c.t) + kd.div(c.t + k - 1);
            if (k > 1 && c.t != kd.div(c.t) * k && c.d < p.out_cap)
                static_cast<int *>(p.out)[c.d] = 1 << (2 * k);  // UNK tail
        }
        for (long long i = 0; i < nbz; ++i) {
            const long long g = c.nb + i;
            if (g < p.offsets_cap) p.offsets_out[g] = tclose;
        }
    }
    if (p.totals_out) {
        p.totals_out[0] = incl.nb > 0 ? incl.d : 0;
        p.totals_out[1] = incl.nb > 0 ? incl.nb - 1 : 0;
    }
    if (p.carry_out) {
        Carry o;
        o.a = incl;
        o.hstate = p.carry_in ? p.carry_in->hstate : HS_LS;
        o.pad = 0;
        *p.carry_out = o;
    }
}

template <int MODE>
cudaError_t launch_mode(int bsrc, const TileParams &p, const LaunchShape &sh, cudaStream_t s,
                        int sm_count);

bool tile_shape_supported(const LaunchShape &sh) {
    return (sh.tile == 8192 && sh.threads == 256 && sh.chunk_tiles == 8) ||
           (sh.tile == 16384 && sh.threads == 256 && (sh.chunk_tiles == 4 || sh.chunk_tiles == 8)) ||
           (sh.tile == 32768 && sh.threads == 512 && sh.chunk_tiles == 4);
}

cudaError_t launch_tile_kernel(int mode, int bsrc, const TileParams &p, const LaunchShape &sh,
                               cudaStream_t s, int sm_count) {
    switch (mode) {
    case MODE_CHAR: return launch_mode<MODE_CHAR>(bsrc, p, sh, s, sm_count);
    case MODE_KMER: return launch_mode<MODE_KMER>(bsrc, p, sh, s, sm_count);
    case MODE_SYM: return launch_mode<MODE_SYM>(bsrc, p, sh, s, sm_count);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_empty_chunk(const TileParams &p, int list_source, cudaStream_t s) {
    empty_chunk_kernel<<<1, 32, 0, s>>>(p, list_source);
    return cudaGetLastError();
}

}  // namespace dnatok
