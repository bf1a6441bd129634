// noalloc.cu -- dnatok_encode_kmer_noalloc: the k-mer encode for callers that
// may not allocate device memory.
//
// Some callers cannot call cudaMalloc: a library that runs inside another
// framework's memory pool, a process whose allocator already owns the whole
// device, or code that must not risk the device-wide synchronization an
// allocation can bring.  This entry point runs the same single-launch k-mer
// kernel as dnatok_encode, but its working memory (the look-back
// descriptors, the chunk counters and the status word) lives in one
// file-scope __device__ array of fixed size instead of a handle's
// allocation.  Every GPU that loads the library holds that array until the
// process exits.
//
// On the host the array's name stands for a host-side stand-in object, not a
// device address, so the first call on each device, with that device
// current, asks the runtime for the address with cudaGetSymbolAddress and
// caches it.  That first call should come before any stream capture.  Every
// call shares the array and finds it as the previous call left it, so each
// call clears on its stream what the kernel needs at zero; calls whose work
// overlaps on the GPU race with each other.
#include <cstring>
#include <mutex>

#include "tile_kernel.cuh"
#include "internal.h"

namespace dnatok {
namespace {

// Largest input one call accepts, and the chunk shape it is launched with.
constexpr long long kNoallocMaxBytes = DNATOK_NOALLOC_MAX_BYTES;
constexpr int kNoallocTile = 16384, kNoallocThreads = 256, kNoallocChunkTiles = 8;
constexpr long long kNoallocChunks =
    (kNoallocMaxBytes + 15 + (long long)kNoallocTile * kNoallocChunkTiles - 1) /
        ((long long)kNoallocTile * kNoallocChunkTiles) + 1;

struct NoallocScratch {
    unsigned long long counter[2];  // chunk claim / exit counters
    int status;                     // device-side error word
    int pad[27];
    TileDesc desc[kNoallocChunks];  // one look-back descriptor per chunk
};

__device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoallocScratch *g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// Runs after the tile kernel: a recorded device-side error turns the totals
// into {-1, -1}, so a caller without a handle can see it.
__global__ void noalloc_finish_kernel(const int *status, long long *totals) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *status != 0) {
        totals[0] = -1;
        totals[1] = -1;
    }
}

dnatok_status setup_device(int dev, NoallocScratch **out, int *sms) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
            return DNATOK_ERR_CUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return DNATOK_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<NoallocScratch *>(ptr);
        g_sm_count[dev] = n;
    }
    *out = g_scratch_ptr[dev];
    *sms = g_sm_count[dev];
    return DNATOK_OK;
}

}  // namespace
}  // namespace dnatok

using namespace dnatok;

extern "C" DNATOK_API dnatok_status dnatok_encode_kmer_noalloc(
    int k, const uint8_t *bytes_d, int64_t n_bytes, const int64_t *seq_offsets_d, int64_t n_seq,
    int32_t *ids_out_d, int64_t ids_capacity, int64_t *id_offsets_d, int64_t offsets_capacity,
    int64_t *totals_d, dnatok_cuda_stream stream) {
    if (k < 1 || k > DNATOK_MAX_K) return DNATOK_ERR_ARG;
    if (n_bytes < 0 || (n_bytes > 0 && !bytes_d) || !seq_offsets_d || n_seq < 0 || !id_offsets_d)
        return DNATOK_ERR_ARG;
    if (n_bytes > kNoallocMaxBytes) return DNATOK_ERR_CAPACITY;  // beyond the fixed scratch
    if (n_seq == 0 && n_bytes != 0) return DNATOK_ERR_ARG;
    if (n_seq >= INT32_MAX - 1 || offsets_capacity < n_seq + 1) return DNATOK_ERR_CAPACITY;
    long long need = n_bytes;
    if (k > 1) {
        const long long alt = (n_bytes + n_seq * (long long)(k - 1)) / k;
        if (alt < need) need = alt;
    }
    if (ids_capacity < need || (need > 0 && !ids_out_d)) return DNATOK_ERR_CAPACITY;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DNATOK_ERR_CUDA;
    NoallocScratch *scratch = nullptr;
    int sms = 0;
    dnatok_status st = setup_device(dev, &scratch, &sms);
    if (st != DNATOK_OK) return st;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int head_pad = (int)((uintptr_t)bytes_d & 15u);
    const long long n_tiles = (head_pad + n_bytes + kNoallocTile - 1) / kNoallocTile;
    const long long n_chunks = (n_tiles + kNoallocChunkTiles - 1) / kNoallocChunkTiles;
    // Everything the kernel expects to start at zero: counters, status, and
    // the descriptors this call will use (so epoch 1 is always fresh).
    const size_t clear = offsetof(NoallocScratch, desc) + sizeof(TileDesc) * (size_t)n_chunks;
    if (cudaMemsetAsync(scratch, 0, clear, s) != cudaSuccess) return DNATOK_ERR_CUDA;

    TileParams p;
    std::memset(&p, 0, sizeof(p));
    p.bytes = bytes_d;
    p.n_bytes = n_bytes;
    p.seq_offsets = reinterpret_cast<const long long *>(seq_offsets_d);
    p.n_bnd = n_seq + 1;
    p.out = ids_out_d;
    p.out_cap = ids_capacity;
    p.offsets_out = reinterpret_cast<long long *>(id_offsets_d);
    p.offsets_cap = offsets_capacity;
    p.totals_out = reinterpret_cast<long long *>(totals_d);
    p.desc = scratch->desc;
    p.tile_counter = scratch->counter;
    p.status = &scratch->status;
    p.k = k;
    p.head_pad = head_pad;
    p.lut_keeps_bases = 1;
    p.spin_limit = kSpinLimit;
    p.skip_chunk = -1;
    p.epoch = 1;
    cudaError_t e;
    if (n_bytes == 0) {
        e = launch_empty_chunk(p, 1, s);
    } else {
        p.n_tiles = n_tiles;
        p.n_chunks = n_chunks;
        LaunchShape sh{kNoallocTile, kNoallocThreads, 4, kNoallocChunkTiles};
        e = launch_tile_kernel(MODE_KMER, 0 /* list boundaries */, p, sh, s, sms);
    }
    if (e != cudaSuccess) return DNATOK_ERR_CUDA;
    if (totals_d) {
        noalloc_finish_kernel<<<1, 32, 0, s>>>(&scratch->status, p.totals_out);
        if (cudaGetLastError() != cudaSuccess) return DNATOK_ERR_CUDA;
    }
    return DNATOK_OK;
}
