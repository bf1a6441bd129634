// shard.cu -- byte-balanced contiguous record shards for one process per
// GPU.  Records are independent, so each rank encodes its own range with no
// exchange on the data path; the only cross-rank step is the exclusive scan
// of per-shard id counts that turns local id offsets into global ones, done
// by the caller's collective.  Host code only.
#include <cstdint>

#include "dnatok.h"

extern "C" {

dnatok_status dnatok_shard_records(const int64_t *seq_offsets_host, int64_t n_seq,
                                   int32_t world_size, int64_t *bounds_out) {
    if (!seq_offsets_host || !bounds_out || n_seq < 0 || world_size < 1) return DNATOK_ERR_ARG;
    if (seq_offsets_host[0] != 0) return DNATOK_ERR_ARG;
    for (int64_t r = 0; r < n_seq; ++r)
        if (seq_offsets_host[r + 1] < seq_offsets_host[r]) return DNATOK_ERR_ARG;
    const int64_t n_bytes = seq_offsets_host[n_seq];
    bounds_out[0] = 0;
    for (int32_t i = 1; i < world_size; ++i) {
        // the first record starting at or after i * n_bytes / world_size
        // (a record that spans the split point stays with the earlier shard)
        const int64_t p = (int64_t)((__int128)n_bytes * i / world_size);
        int64_t lo = bounds_out[i - 1], hi = n_seq;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (seq_offsets_host[mid] >= p) hi = mid; else lo = mid + 1;
        }
        bounds_out[i] = lo;
    }
    bounds_out[world_size] = n_seq;
    return DNATOK_OK;
}

}  // extern "C"
