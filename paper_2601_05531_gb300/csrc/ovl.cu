// ovl.cu -- overlapping k-mers with stride 1: every window of k consecutive
// kept bases of a record is a token, adjacent tokens share k - 1 bases, and a
// record of L kept bases gives max(0, L - k + 1) tokens (Sec. 1.1 and
// Table 1: "overlapping k-mer tokenization with stride 1" yields L - k + 1
// tokens).  Ids are the closed form of the non-overlapping mode,
// sum_i 4^(k-1-i) * code(b_i) with A0 C1 G2 T3, and UNK = 4^k for a window
// holding an N-class base.
//
// Three launches per encode:
//   1. the symbol pass (the tile kernel in MODE_SYM, or its direct path): one
//      byte per kept base (0..3, 4 for N-class) and the record starts in
//      symbols, written to the caller's id_offsets (FASTA headers and
//      separators already removed);
//   2. ovl_offsets_kernel (one block): copies those starts to the handle's
//      workspace and rewrites id_offsets in place with the token offsets;
//   3. ovl_emit_kernel: each CTA walks a contiguous run of 4096-symbol tiles,
//      staging the tile's symbols (plus k - 1) and a window of its records
//      in shared memory; consecutive threads write consecutive ids.
#include <cstring>

#include "handle.h"
#include "tile_kernel.cuh"

struct OvlState {
    uint8_t *d_sym = nullptr;   // one symbol per kept base
    long long cap_sym = 0;
    long long *d_srec = nullptr;  // record starts in symbols (n_rec + 1)
    long long cap_srec = 0;
    long long *d_tot = nullptr;   // {symbols, records} of the symbol pass
};

namespace {

constexpr int kOT = 4096;          // symbols per emit tile
constexpr int kOThreads = 256;
constexpr int kORW = 64;           // records of a tile kept in shared memory
constexpr int kOPlanThreads = 1024;
constexpr int kOPlanTile = 4096;   // records per pass of the offsets kernel

__device__ __forceinline__ long long ovl_tokens(long long L, int k) { return L >= k ? L - k + 1 : 0; }

// Largest r in [0, n_rec - 1] with srec[r] <= j (srec sorted, srec[0] = 0),
// by one thread.
__device__ long long ovl_find(const long long *srec, long long n_rec, long long j) {
    long long lo = 0, hi = n_rec - 1;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (srec[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Token offsets from the symbol pass's record starts, in place.
__global__ void __launch_bounds__(kOPlanThreads) ovl_offsets_kernel(long long *offs, long long *srec,
                                                                    const long long *tot, int k,
                                                                    long long *totals_out) {
    constexpr int kPer = kOPlanTile / kOPlanThreads;
    __shared__ long long s_v[kOPlanTile + 1];
    __shared__ long long wsum[kOPlanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = tot[1];  // records
    long long carry = 0;
    for (long long r0 = 0; r0 < n; r0 += kOPlanTile) {
        const int cnt = (n - r0 < kOPlanTile) ? (int)(n - r0) : kOPlanTile;
        // read this pass's starts (and the next pass's first) before any is
        // overwritten; keep a copy for the emit kernel
        for (int i = tid; i <= cnt; i += kOPlanThreads) {
            const long long v = offs[r0 + i];
            s_v[i] = v;
            if (i < cnt) srec[r0 + i] = v;
        }
        __syncthreads();
        long long t[kPer], sum = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int i = tid * kPer + j;
            t[j] = i < cnt ? ovl_tokens(s_v[i + 1] - s_v[i], k) : 0;
            sum += t[j];
        }
        long long x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        long long pre = carry, tt = 0;
        for (int w = 0; w < kOPlanThreads / 32; ++w) {
            if (w < warp) pre += wsum[w];
            tt += wsum[w];
        }
        long long run = pre + x - sum;
        __syncthreads();  // every s_v read above is done
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            s_v[tid * kPer + j] = run;
            run += t[j];
        }
        __syncthreads();
        for (int i = tid; i < cnt; i += kOPlanThreads) offs[r0 + i] = s_v[i];
        carry += tt;
        __syncthreads();
    }
    if (tid == 0) {
        srec[n] = offs[n];  // the symbol count (not overwritten above)
        offs[n] = carry;
        if (totals_out) {
            totals_out[0] = carry;
            totals_out[1] = n;
        }
    }
}

template <int K>
__global__ void __launch_bounds__(kOThreads) ovl_emit_kernel(const uint8_t *sym, const long long *srec,
                                                             const long long *offs, const long long *tot,
                                                             int *out, long long ids_cap) {
    constexpr unsigned UNK = 1u << (2 * K);
    __shared__ uint8_t s_sym[kOT + 16];
    __shared__ long long s_rs[kORW + 1], s_ob[kORW];
    __shared__ long long s_rb;
    __shared__ int s_nw;
    const int tid = threadIdx.x;
    const long long n_sym = tot[0], n_rec = tot[1];
    if (n_rec < 1 || n_sym < 1) return;
    const long long n_tiles = (n_sym + kOT - 1) / kOT;
    const long long t_begin = (long long)blockIdx.x * n_tiles / gridDim.x;
    const long long t_end = (long long)(blockIdx.x + 1) * n_tiles / gridDim.x;
    for (long long tile = t_begin; tile < t_end; ++tile) {
        const long long j0 = tile * kOT;
        const long long j1 = (j0 + kOT < n_sym) ? j0 + kOT : n_sym;
        const long long jh = (j1 + K - 1 < n_sym) ? j1 + K - 1 : n_sym;
        for (long long i = tid; i < jh - j0; i += kOThreads) s_sym[i] = sym[j0 + i];
        if (tid == 0) {
            // the record holding j0: from the last tile's window when it is there
            long long rb;
            if (tile > t_begin && s_rs[0] <= j0 && (s_rb + s_nw >= n_rec || s_rs[s_nw] > j0)) {
                int i = 0;
                while (i + 1 < s_nw && s_rs[i + 1] <= j0) ++i;
                rb = s_rb + i;
            } else {
                rb = ovl_find(srec, n_rec, j0);
            }
            s_rb = rb;
            s_nw = (n_rec - rb < kORW) ? (int)(n_rec - rb) : kORW;
        }
        __syncthreads();
        const long long rb = s_rb;
        const int nw = s_nw;
        for (int l = tid; l <= nw; l += kOThreads) {
            s_rs[l] = srec[rb + l];
            if (l < nw) s_ob[l] = offs[rb + l];
        }
        __syncthreads();
        int i = 0;  // this thread's window record (its j only grow)
        for (long long j = j0 + tid; j < j1; j += kOThreads) {
            while (i + 1 < nw && s_rs[i + 1] <= j) ++i;
            long long rs, re, ob;
            if (i + 1 == nw && rb + nw < n_rec && s_rs[nw] <= j) {
                // more records start in this tile than the window holds
                const long long r = ovl_find(srec, n_rec, j);
                rs = srec[r];
                re = srec[r + 1];
                ob = offs[r];
            } else {
                rs = s_rs[i];
                re = s_rs[i + 1];
                ob = s_ob[i];
            }
            if (j + K <= re) {
                const uint8_t *w = s_sym + (j - j0);
                unsigned id = 0, bad = 0;
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    const unsigned c = w[t];
                    id = (id << 2) | (c & 3u);
                    bad |= c & 4u;
                }
                const long long o = ob + (j - rs);
                if (o >= 0 && o < ids_cap) out[o] = (int)(bad ? UNK : id);  // (malformed input)
            }
        }
        __syncthreads();  // the tile's shared memory is reused by the next
    }
}

cudaError_t launch_emit(int k, unsigned grid, const uint8_t *sym, const long long *srec,
                        const long long *offs, const long long *tot, int *out, long long cap,
                        cudaStream_t s) {
    switch (k) {
#define DNATOK_OK_K(KK) \
    case KK: ovl_emit_kernel<KK><<<grid, kOThreads, 0, s>>>(sym, srec, offs, tot, out, cap); break;
        DNATOK_OK_K(1) DNATOK_OK_K(2) DNATOK_OK_K(3) DNATOK_OK_K(4) DNATOK_OK_K(5) DNATOK_OK_K(6)
        DNATOK_OK_K(7) DNATOK_OK_K(8) DNATOK_OK_K(9) DNATOK_OK_K(10) DNATOK_OK_K(11)
        DNATOK_OK_K(12) DNATOK_OK_K(13) DNATOK_OK_K(14) DNATOK_OK_K(15)
#undef DNATOK_OK_K
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

void free_ovl(OvlState *o) {
    cudaFree(o->d_sym);
    cudaFree(o->d_srec);
    cudaFree(o->d_tot);
    o->d_sym = nullptr;
    o->d_srec = nullptr;
    o->d_tot = nullptr;
    o->cap_sym = o->cap_srec = 0;
}

}  // namespace

namespace dnatok {

void ovl_destroy(dnatok_handle *h) {
    if (!h->ovl) return;
    free_ovl(h->ovl);
    delete h->ovl;
    h->ovl = nullptr;
}

dnatok_status ovl_reserve(dnatok_handle *h, long long max_bytes, long long max_offsets,
                          cudaStream_t s) {
    if (!h->ovl) {
        h->ovl = new (std::nothrow) OvlState();
        if (!h->ovl) return fail(h, DNATOK_ERR_NOMEM, "host allocation failed");
    }
    OvlState *o = h->ovl;
    if (max_bytes <= o->cap_sym && max_offsets <= o->cap_srec && o->d_tot) return DNATOK_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(h, DNATOK_ERR_STATE,
                    "the workspace must grow during stream capture; call dnatok_reserve first");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaDeviceSynchronize");
    const long long cs_ = max_bytes > o->cap_sym ? max_bytes + max_bytes / 8 + 4096 : o->cap_sym;
    const long long cr = max_offsets > o->cap_srec ? max_offsets + max_offsets / 8 + 64 : o->cap_srec;
    free_ovl(o);
    e = cudaMalloc(&o->d_sym, (size_t)cs_ + 16);
    if (e == cudaSuccess) e = cudaMalloc(&o->d_srec, sizeof(long long) * (size_t)(cr + 1));
    if (e == cudaSuccess) e = cudaMalloc(&o->d_tot, 2 * sizeof(long long));
    if (e != cudaSuccess) {
        free_ovl(o);
        return fail_cuda(h, e, "cudaMalloc(overlapping k-mer workspace)");
    }
    o->cap_sym = cs_;
    o->cap_srec = cr;
    return DNATOK_OK;
}

dnatok_status ovl_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                         const int64_t *seq_offsets_d, int64_t n_seq, int32_t *ids_out_d,
                         int64_t ids_capacity, int64_t *id_offsets_d, int64_t offsets_capacity,
                         int64_t *totals_d, cudaStream_t s) {
    dnatok_status st = ovl_reserve(h, n_bytes, offsets_capacity, s);
    if (st != DNATOK_OK) return st;
    OvlState *o = h->ovl;
    const bool raw = (h->fmt == DNATOK_RAW);
    // 1. symbols and record starts (in symbols)
    st = run_tile_encode(h, MODE_SYM, 1, raw ? BSRC_LIST : BSRC_FASTA, bytes_d, n_bytes,
                         reinterpret_cast<const long long *>(seq_offsets_d), raw ? n_seq + 1 : 0,
                         o->d_sym, o->cap_sym, reinterpret_cast<long long *>(id_offsets_d),
                         offsets_capacity, o->d_tot, nullptr, nullptr, raw ? 0 : 1, raw ? 0 : 1, s);
    if (st != DNATOK_OK) return st;
    // 2. token offsets
    ovl_offsets_kernel<<<1, kOPlanThreads, 0, s>>>(reinterpret_cast<long long *>(id_offsets_d),
                                                    o->d_srec, o->d_tot, h->k,
                                                    reinterpret_cast<long long *>(totals_d));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e, "overlap offsets launch");
    // 3. ids
    long long tiles = (n_bytes + kOT - 1) / kOT;
    long long grid = (long long)h->sm_count * 8;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    e = launch_emit(h->k, (unsigned)grid, o->d_sym, o->d_srec,
                    reinterpret_cast<const long long *>(id_offsets_d), o->d_tot, ids_out_d,
                    ids_capacity, s);
    if (e != cudaSuccess) return fail_cuda(h, e, "overlap emit launch");
    return DNATOK_OK;
}

}  // namespace dnatok
