// search.cuh -- searches over sorted int64 offset arrays by one warp.
#pragma once

namespace dnatok {

// Largest r in [0, n - 1] with a[r] <= x, for a non-decreasing a with
// a[0] <= x and n >= 1.  Called by all 32 lanes of a warp (each gets the
// result).  Every round the lanes probe 32 evenly spaced points of the
// current range [lo, hi] at once and keep the part after the last probe that
// is still <= x, so the range shrinks 32-fold per round of memory latency
// (three rounds for 4096 entries) instead of 2-fold.
__device__ __forceinline__ long long warp_find_le(const long long *a, long long n, long long x) {
    const int lane = threadIdx.x & 31;
    long long lo = 0, hi = n - 1;
    while (lo < hi) {
        const long long span = hi - lo;
        const long long p = lo + (span * (lane + 1) >> 5);
        const unsigned ok = __ballot_sync(0xffffffffu, a[p] <= x);
        const int c = __popc(ok);  // the probes <= x form a prefix of the lanes
        const long long pc1 = __shfl_sync(0xffffffffu, p, c > 0 ? c - 1 : 0);
        const long long pc = __shfl_sync(0xffffffffu, p, c < 32 ? c : 31);
        if (c == 0) {
            hi = pc1 - 1;  // (pc1 = the first probe, above lo)
        } else {
            lo = pc1;
            if (c < 32) hi = pc - 1;
        }
    }
    return lo;
}

// First r in [0, n] with a[r] >= x, for a non-decreasing a of n + 1 entries.
// Called by all 32 lanes of a warp.
__device__ __forceinline__ long long warp_first_ge(const long long *a, long long n, long long x) {
    if (a[0] >= x) return 0;
    return warp_find_le(a, n + 1, x - 1) + 1;
}

}  // namespace dnatok
