// ovl.cu -- the modes built on the symbol pass: overlapping k-mers (a window
// at every position) and table-driven k-mers.
//
// Overlapping k-mers: every window of k consecutive kept bases of a record is
// a token, neighbours overlapping in all but one base, and a record of L kept
// bases gives max(0, L - k + 1) tokens (Sec. 1.1 and Table 1 give the
// L - k + 1 count).  Ids are the closed
// form of the non-overlapping mode, sum_i 4^(k-1-i) * code(b_i) with A0 C1 G2
// T3, and UNK = 4^k for a window holding an N-class base.  Three launches:
//   1. the symbol pass (the tile kernel in MODE_SYM, or its direct path): one
//      byte per kept base (0..3, 4 for N-class) and the record starts in
//      symbols, written to the caller's id_offsets (FASTA headers and
//      separators already removed);
//   2. offsets_kernel<kOffsetsTokens> (one block): copies those starts to the
//      handle's workspace and rewrites id_offsets in place with the token
//      offsets;
//   3. ovl_emit_kernel: each CTA walks a contiguous run of 4096-symbol tiles,
//      staging the tile's symbols (plus k - 1) and a window of its records
//      in shared memory; consecutive threads write consecutive ids.
//
// Table-driven k-mers (Algorithm 1 builds kmer_lut[0..5^k-1] over base-5
// digits, Algorithm 2 applies it as MapKmer): the symbols of a record are cut
// into windows of k from its start; a whole window emits kmer_lut[index] or,
// when that entry is -1, its k symbols through base_ids; a tail of L mod k
// symbols goes through base_ids.  A window's token count (1, k or the tail
// length) depends on the table, so the positions need a scan:
//   1. the symbol pass, as above;
//   2. offsets_kernel<kOffsetsWindows>: record starts to the workspace and
//      the window offsets wpre[r] = sum of ceil(L / k) over earlier records;
//   3. ktab_tile_kernel<K, false>: per tile of 2048 windows, its token count;
//   4. tile_scan_kernel (one block): exclusive scan of the tile counts, the
//      totals and the offsets of records with no window left;
//   5. ktab_tile_kernel<K, true>: recounts, scans inside the block and writes
//      the ids and the record offsets.
// For k <= 6 with every id below 0xFFFF the table is held in each CTA's
// shared memory as u16 (a blocked 6-mer vocabulary takes 31 KB).
#include <atomic>
#include <cstring>

#include "handle.h"
#include "search.cuh"
#include "tile_kernel.cuh"
#include "ktab.cuh"

struct OvlState {
    uint8_t *d_sym = nullptr;   // one symbol per kept base
    long long cap_sym = 0;
    long long *d_srec = nullptr;  // record starts in symbols (n_rec + 1)
    long long *d_wpre = nullptr;  // table-driven k-mers: window offsets (n_rec + 1)
    long long cap_srec = 0;
    long long *d_tot = nullptr;   // {symbols, records} of the symbol pass
    long long *d_tsum = nullptr;  // table-driven k-mers: per-tile token counts
    long long cap_tsum = 0;
    // table-driven k-mers straight from RAW bytes: per tile of windows its
    // first window's record, and per window its entry (sized for cap_sym
    // input bytes and cap_srec records; the tile counts go to d_tsum)
    long long *d_trec = nullptr;
    void *d_went = nullptr;
};

namespace {

using namespace dnatok;

constexpr int kOT = 4096;          // symbols per emit tile
constexpr int kOThreads = 256;
constexpr int kOPlanThreads = 1024;
constexpr int kOPlanTile = 4096;   // records per pass of the offsets kernel

__device__ __forceinline__ long long ovl_tokens(long long L, int k) { return L >= k ? L - k + 1 : 0; }

// Stage sym[j0 .. j0 + n) in shared memory as the 16-byte aligned span
// around it, s[x] = sym[(j0 & ~15) + x] for x < (j0 & 15) + n rounded up to
// 16, with 16-byte loads issued together.
// The symbol buffer is 16-byte aligned and has 16 spare bytes at its end, so
// the rounded span stays inside it.  Returns j0 & 15, the shift of j0 in s.
__device__ __forceinline__ int stage_symbols(uint8_t *s, const uint8_t *sym, long long j0, long long n,
                                             int tid, int nthreads) {
    const int lead = (int)(j0 & 15);
    const uint4 *src = reinterpret_cast<const uint4 *>(sym + (j0 - lead));
    uint4 *dst = reinterpret_cast<uint4 *>(s);
    const int chunks = (int)((lead + n + 15) >> 4);
#pragma unroll 4
    for (int c = tid; c < chunks; c += nthreads) dst[c] = src[c];
    return lead;
}

enum { kOffsetsTokens = 0, kOffsetsWindows = 1 };

// From the symbol pass's record starts (offs, n_rec + 1 entries): copy them
// to srec and write, for every record, the running sum of f(L) over earlier
// records -- f(L) = max(0, L - k + 1) tokens in place into offs
// (kOffsetsTokens), or ceil(L / k) windows into wpre (kOffsetsWindows).  If
// the records found do not fit offs_cap entries the pass records
// DEV_CAPACITY, zeroes the symbol pass's record count (so the later kernels
// do nothing) and reports {0, n_rec} in totals_out.
template <int KIND>
__global__ void __launch_bounds__(kOPlanThreads) offsets_kernel(long long *offs, long long *srec,
                                                                long long *wpre, long long *tot,
                                                                int k, long long offs_cap,
                                                                long long *totals_out, int *status,
                                                                const unsigned *gate,
                                                                unsigned gate_epoch) {
    constexpr int kPer = kOPlanTile / kOPlanThreads;
    __shared__ long long s_v[kOPlanTile + 1];
    __shared__ long long wsum[kOPlanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (gate && *(volatile const unsigned *)gate != gate_epoch) return;  // the direct path did it
    const long long n = tot[1];  // records
    if (n + 1 > offs_cap) {
        __syncthreads();  // every thread has read tot[1]
        if (tid == 0) {
            tot[1] = 0;
            set_dev_status(status, DEV_CAPACITY);
            if (totals_out) {
                totals_out[0] = 0;
                totals_out[1] = n;
            }
        }
        return;
    }
    long long *dst = KIND == kOffsetsTokens ? offs : wpre;
    long long carry = 0;
    for (long long r0 = 0; r0 < n; r0 += kOPlanTile) {
        const int cnt = (n - r0 < kOPlanTile) ? (int)(n - r0) : kOPlanTile;
        // read this pass's starts (and the next pass's first) before any is
        // overwritten; keep a copy for the later kernels
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
            long long f = 0;
            if (i < cnt) {
                const long long L = s_v[i + 1] - s_v[i];
                f = KIND == kOffsetsTokens ? ovl_tokens(L, k) : (L + k - 1) / k;
            }
            t[j] = f;
            sum += f;
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
        for (int i = tid; i < cnt; i += kOPlanThreads) dst[r0 + i] = s_v[i];
        carry += tt;
        __syncthreads();
    }
    if (tid == 0) {
        srec[n] = offs[n];  // the symbol count (not overwritten above)
        dst[n] = carry;
        if (KIND == kOffsetsTokens && totals_out) {
            totals_out[0] = carry;
            totals_out[1] = n;
        }
    }
}

// Overlapping k-mer ids, warp by warp (no block barrier): each warp takes a
// contiguous run of 512-symbol tiles.  Per tile a lane loads its 16 symbols
// (and the next lane's by shuffle, for the k - 1 symbols a window reaches
// past them), slides a 2-bit window over them remembering the last N-class
// symbol, and writes its 16 ids to the warp's rows in shared memory (17 ints
// per row, so neighbouring lanes hit different banks).  The starts of a record
// that have a token (j + k <= record end) are contiguous with contiguous
// output slots: when the whole tile is such a run the warp writes it as 16
// rows of 32 consecutive ids (every store a full 128-byte line whatever the
// alignment), otherwise record by record.  A register cursor follows the
// records from tile to tile.
constexpr int kOWT = 512;  // symbols per warp tile

template <int K>
__global__ void __launch_bounds__(kOThreads) ovl_emit_kernel(const uint8_t *sym, const long long *srec,
                                                             const long long *offs, const long long *tot,
                                                             int *out, long long ids_cap) {
    constexpr unsigned UNK = 1u << (2 * K);
    constexpr unsigned MASK = UNK - 1u;
    constexpr int kW = kOThreads / 32;
    __shared__ int s_id[kW][32 * 17];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long n_sym = tot[0], n_rec = tot[1];
    if (n_rec < 1 || n_sym < 1) return;
    const long long n_wt = (n_sym + kOWT - 1) / kOWT;
    const long long nw = (long long)gridDim.x * kW, gw = (long long)blockIdx.x * kW + warp;
    const long long t_begin = gw * n_wt / nw, t_end = (gw + 1) * n_wt / nw;
    if (t_begin >= t_end) return;
    int *const rows = s_id[warp];
    // the record cursor: r holds symbol rs .. re - 1, its first id at ob
    long long r = ovl_find(srec, n_rec, t_begin * kOWT);
    long long rs = srec[r], re = srec[r + 1], ob = offs[r];
    // the symbol buffer has spare bytes past the last tile: every load below
    // stays inside it; the next tile's vector is loaded one tile ahead, and its
    // lane 0 gives lane 31 the symbols past this tile
    uint4 vn = *reinterpret_cast<const uint4 *>(sym + t_begin * kOWT + 16 * lane);
    for (long long t = t_begin; t < t_end; ++t) {
        const long long j0 = t * kOWT;
        const uint4 v = vn;
        vn = *reinterpret_cast<const uint4 *>(sym + j0 + kOWT + 16 * lane);
        uint4 nx, n0;
        nx.x = __shfl_down_sync(0xffffffffu, v.x, 1);
        nx.y = __shfl_down_sync(0xffffffffu, v.y, 1);
        nx.z = __shfl_down_sync(0xffffffffu, v.z, 1);
        nx.w = __shfl_down_sync(0xffffffffu, v.w, 1);
        n0.x = __shfl_sync(0xffffffffu, vn.x, 0);
        n0.y = __shfl_sync(0xffffffffu, vn.y, 0);
        n0.z = __shfl_sync(0xffffffffu, vn.z, 0);
        n0.w = __shfl_sync(0xffffffffu, vn.w, 0);
        if (lane == 31) nx = n0;
        {
            const unsigned wd[8] = {v.x, v.y, v.z, v.w, nx.x, nx.y, nx.z, nx.w};
            unsigned id = 0;
            int last_n = -1000;  // position of the last N-class symbol
            int *row = rows + lane * 17;
#pragma unroll
            for (int p = 0; p < 16 + K - 1; ++p) {
                const unsigned c = (wd[p >> 2] >> (8 * (p & 3))) & 0xFFu;
                id = ((id << 2) | (c & 3u)) & MASK;
                if (c >= 4u) last_n = p;
                if (p >= K - 1) row[p - (K - 1)] = (last_n > p - K) ? (int)UNK : (int)id;
            }
        }
        __syncwarp();
        while (re <= j0 && r + 1 < n_rec) {  // (warp-uniform)
            ++r;
            rs = re;
            re = srec[r + 1];
            ob = offs[r];
        }
        if (rs <= j0 && j0 + kOWT + K - 1 <= re && ob + (j0 - rs) + kOWT <= ids_cap) {
            // the whole tile is one run of starts with tokens
            int *dst = out + ob + (j0 - rs);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int x = 32 * i + lane;
                dst[x] = rows[(x >> 4) * 17 + (x & 15)];
            }
        } else {
            // record by record: the starts of record q with a token in this
            // tile are [max(qs, j0), min(qe - K + 1, j0 + kOWT))
            long long q = r, qs = rs, qe = re, qb = ob;
            while (true) {
                const long long a = qs > j0 ? qs : j0;
                const long long b = (qe - K + 1 < j0 + kOWT) ? qe - K + 1 : j0 + kOWT;
                if (b > a) {
                    const long long oa = qb + (a - qs);
                    for (long long y = lane; y < b - a; y += 32) {
                        const int x = (int)(a - j0 + y);
                        if (oa + y < ids_cap) out[oa + y] = rows[(x >> 4) * 17 + (x & 15)];
                    }
                }
                if (qe >= j0 + kOWT || q + 1 >= n_rec) break;
                ++q;
                qs = qe;
                qe = srec[q + 1];
                qb = offs[q];
            }
        }
        __syncwarp();  // the rows are rewritten by the next tile
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

// One tile of windows [w0, w1): count (EMIT = false: the tile's token count
// to tsum[tile]) or emit (EMIT = true: ids from tsum[tile], by then the
// tile's exclusive token offset, and the record offsets of records whose
// first window is here).  Each thread takes kKPer consecutive windows; the
// emit recounts them after the block scan instead of keeping them in
// registers, assembles the tile's ids in shared memory when they fit, and
// writes them out in aligned 16-byte stores.  T16: the ids table lives in
// shared memory as u16 (k <= 6, every id below 0xFFFF, 0xFFFF = no entry),
// loaded once per CTA; otherwise each window reads kmer_lut from global
// memory.
template <int K, bool EMIT, bool T16>
__global__ void __launch_bounds__(kKThreads) ktab_tile_kernel(
    const uint8_t *sym, const long long *srec, const long long *wpre, const long long *tot,
    const int *klut, const uint16_t *klut16, KtabIds base, long long *tsum, int *out,
    long long ids_cap, long long *id_offsets, const unsigned *gate, unsigned gate_epoch) {
    extern __shared__ __align__(16) uint8_t dyn[];
    uint16_t *s_tab = reinterpret_cast<uint16_t *>(dyn);
    uint8_t *s_sym = dyn + ktab_tab_bytes(K, T16);
    int *s_tok = reinterpret_cast<int *>(dyn + ktab_tab_bytes(K, T16) + ktab_sym_bytes(K));
    __shared__ long long s_wp[kKRW + 1], s_sr[kKRW + 1];
    __shared__ long long s_rb, s_jlo, s_jhi;
    __shared__ int s_nw;
    __shared__ int s_wsum[kKThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (gate && *(volatile const unsigned *)gate != gate_epoch) return;  // the direct path did it
    const long long n_rec = tot[1];
    if (n_rec < 1) return;
    if (T16) {
        const uint4 *src = reinterpret_cast<const uint4 *>(klut16);
        uint4 *dst = reinterpret_cast<uint4 *>(s_tab);
        for (int c = tid; c < ktab_tab_bytes(K, T16) / 16; c += kKThreads) dst[c] = src[c];
        // (ordered before the first read by the barrier after the staging below)
    }
    const long long n_win = wpre[n_rec];
    const long long n_sym = srec[n_rec];
    const long long n_tiles = (n_win + kKW - 1) / kKW;
    // a contiguous run of tiles per CTA, so the shared record window of one
    // tile usually covers the next
    const long long t_begin = (long long)blockIdx.x * n_tiles / gridDim.x;
    const long long t_end = (long long)(blockIdx.x + 1) * n_tiles / gridDim.x;
    for (long long tile = t_begin; tile < t_end; ++tile) {
        const long long w0 = tile * kKW;
        const long long w1 = (w0 + kKW < n_win) ? w0 + kKW : n_win;
        // (the previous tile ended with a barrier: every thread sees the same window)
        const bool reuse = tile > t_begin && s_wp[0] <= w0 &&
                           (s_rb + s_nw >= n_rec || s_wp[s_nw] > w1);
        long long rb, jlo, jhi;
        int nw;
        if (reuse) {
            // the symbols of w0 and w1 from the window, in every thread
            rb = s_rb;
            nw = s_nw;
            int i0 = 0;
            while (i0 + 1 < nw && s_wp[i0 + 1] <= w0) ++i0;
            jlo = s_sr[i0] + (w0 - s_wp[i0]) * K;
            if (w1 >= n_win) {
                jhi = n_sym;
            } else {
                int i1 = i0;
                while (i1 + 1 < nw && s_wp[i1 + 1] <= w1) ++i1;
                jhi = s_sr[i1] + (w1 - s_wp[i1]) * K;
            }
        } else {
            // the records holding w0 and w1 (one warp each), then the window
            if (warp == 0) {
                const long long r0 = warp_find_le(wpre, n_rec, w0);
                if (lane == 0) {
                    s_rb = r0;
                    s_jlo = srec[r0] + (w0 - wpre[r0]) * K;
                }
            } else if (warp == 1) {
                if (w1 >= n_win) {
                    if (lane == 0) s_jhi = n_sym;
                } else {
                    const long long r1 = warp_find_le(wpre, n_rec, w1);
                    if (lane == 0) s_jhi = srec[r1] + (w1 - wpre[r1]) * K;
                }
            }
            __syncthreads();
            rb = s_rb;
            jlo = s_jlo;
            jhi = s_jhi;
            nw = (n_rec - rb < kKRW) ? (int)(n_rec - rb) : kKRW;
            for (int l = tid; l <= nw; l += kKThreads) {
                s_wp[l] = wpre[rb + l];
                s_sr[l] = srec[rb + l];
            }
            if (tid == 0) s_nw = nw;
        }
        long long nsym = jhi - jlo;
        if (nsym > (long long)kKW * K) nsym = (long long)kKW * K;  // (malformed input)
        if (nsym < 0) nsym = 0;
        const int lead = stage_symbols(s_sym, sym, jlo, nsym, tid, kKThreads);
        __syncthreads();
        const uint8_t *t_sym = s_sym + lead;  // t_sym[x] = sym[jlo + x]

        const long long wt = w0 + (long long)tid * kKPer;
        // more records start in this tile than the shared window holds: the
        // general per-window path (searches past the window)
        const bool dense = rb + nw < n_rec && s_wp[nw] < w1;
        int sum = 0;
        if (!dense) {
            if (wt < w1) {
                KCursor c = kc_init<K>(wt, nw, s_wp, s_sr, jlo);
                const int nq = (int)((w1 - wt < kKPer) ? w1 - wt : kKPer);
                if (nq == kKPer && c.rem >= kKPer * K && c.j >= 0 && c.j + kKPer * K <= nsym) {
                    // all eight windows whole and in one record
                    int ent[kKPer], cn[kKPer], ix[kKPer];
                    ktab_fast_windows<K, T16>(s_sym, lead + c.j, klut, s_tab, ent, cn, ix);
#pragma unroll
                    for (int q = 0; q < kKPer; ++q) sum += cn[q];
                } else {
                    for (int q = 0; q < nq; ++q)
                        sum += kc_window<K, T16>(c, nw, rb, s_sr, jlo, t_sym, nsym, klut, s_tab).cnt;
                }
            }
        } else {
            int i = 0;
            for (int q = 0; q < kKPer; ++q) {
                const long long w = wt + q;
                if (w >= w1) break;
                sum += ktab_window<K, T16>(w, i, nw, rb, n_rec, s_wp, s_sr, wpre, srec, t_sym, jlo,
                                           nsym, klut, s_tab).cnt;
            }
        }
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        if (!EMIT) {
            if (tid == 0) {
                long long tt = 0;
                for (int w = 0; w < kKThreads / 32; ++w) tt += s_wsum[w];
                tsum[tile] = tt;
            }
        } else {
            int loc = x - sum, total = 0;
            for (int w = 0; w < kKThreads / 32; ++w) {
                if (w < warp) loc += s_wsum[w];
                total += s_wsum[w];
            }
            const long long tbase = tsum[tile];
            // staged: ids go to s_tok[shift + loc], shift being the
            // misalignment (in ids) of the tile's first output
            const int shift = (int)((reinterpret_cast<uintptr_t>(out + tbase) >> 2) & 3u);
            const bool staged = total + shift <= kKTok;
            int i = 0;
            KCursor c{0, 0, 0, false};
            if (!dense && wt < w1) c = kc_init<K>(wt, nw, s_wp, s_sr, jlo);
            const bool fast = !dense && wt + kKPer <= w1 && c.rem >= kKPer * K && c.j >= 0 &&
                              c.j + kKPer * K <= nsym;
            if (fast) {
                // all eight windows whole and in one record (as in the count)
                int ent[kKPer], cn[kKPer], ix[kKPer];
                ktab_fast_windows<K, T16>(s_sym, lead + c.j, klut, s_tab, ent, cn, ix);
                if (c.first) {
                    long long r = rb + c.i;
                    const long long pos = tbase + loc;
                    id_offsets[r] = pos;
                    while (r > 0 && wpre[r - 1] == wt) id_offsets[--r] = pos;
                }
#pragma unroll
                for (int q = 0; q < kKPer; ++q) {
                    const long long pos = tbase + loc;
                    if (staged) {
                        int *d = s_tok + shift + loc;
                        if (ent[q] >= 0) {
                            d[0] = ent[q];
                        } else {
                            for (int y = 0; y < K; ++y) {
                                const int dg = t_sym[c.j + q * K + y];
                                d[y] = base.b[dg < 5 ? dg : 4];
                            }
                        }
                    } else if (ent[q] >= 0) {
                        if (pos < ids_cap) out[pos] = ent[q];
                    } else {
                        for (int y = 0; y < K; ++y) {
                            const int dg = t_sym[c.j + q * K + y];
                            if (pos + y < ids_cap) out[pos + y] = base.b[dg < 5 ? dg : 4];
                        }
                    }
                    loc += cn[q];
                }
            }
            for (int q = 0; q < (fast ? 0 : kKPer); ++q) {
                const long long w = wt + q;
                if (w >= w1) break;
                const KWin a = dense ? ktab_window<K, T16>(w, i, nw, rb, n_rec, s_wp, s_sr, wpre,
                                                           srec, t_sym, jlo, nsym, klut, s_tab)
                                     : kc_window<K, T16>(c, nw, rb, s_sr, jlo, t_sym, nsym, klut,
                                                         s_tab);
                if (a.r < 0) continue;
                const long long pos = tbase + loc;
                if (a.t == 0) {
                    // the record's first window: its offset, and that of the
                    // empty records just before it
                    long long r = a.r;
                    id_offsets[r] = pos;
                    while (r > 0 && wpre[r - 1] == w) id_offsets[--r] = pos;
                }
                if (staged) {
                    int *d = s_tok + shift + loc;
                    if (a.cnt == 1 && a.ent >= 0) {
                        d[0] = a.ent;
                    } else {
                        for (int y = 0; y < a.cnt; ++y) {
                            const int dg = t_sym[a.j + y];
                            d[y] = base.b[dg < 5 ? dg : 4];
                        }
                    }
                } else if (a.cnt == 1 && a.ent >= 0) {
                    if (pos < ids_cap) out[pos] = a.ent;
                } else {
                    for (int y = 0; y < a.cnt; ++y) {
                        const int dg = t_sym[a.j + y];
                        if (pos + y < ids_cap) out[pos + y] = base.b[dg < 5 ? dg : 4];
                    }
                }
                loc += a.cnt;
            }
            if (staged) {
                __syncthreads();
                const int span = shift + total;
                int *g = out + (tbase - shift);  // 16-byte aligned
                const long long lim = ids_cap - (tbase - shift);  // ids of g inside the buffer
                for (int c = tid; c < (span + 3) >> 2; c += kKThreads) {
                    const int lo = c * 4, hi = lo + 4;
                    if (lo >= shift && hi <= span && hi <= lim) {
                        *reinterpret_cast<int4 *>(g + lo) = *reinterpret_cast<const int4 *>(s_tok + lo);
                    } else {
                        for (int y = lo > shift ? lo : shift; y < (hi < span ? hi : span); ++y)
                            if (y < lim) g[y] = s_tok[y];
                    }
                }
            }
        }
        __syncthreads();  // shared memory is reused by the next tile
    }
}

// Resident CTAs per SM of one instantiation; the first call also raises its
// dynamic shared memory limit (dnatok_reserve makes that call, so a first
// encode under stream capture finds it done).
template <int K, bool EMIT, bool T16>
cudaError_t ktab_init(int *per_sm_out) {
    constexpr int smem = ktab_smem(K, EMIT, T16);
    static std::atomic<int> per_sm{0};
    if (per_sm.load() == 0) {
        cudaError_t e = cudaFuncSetAttribute(ktab_tile_kernel<K, EMIT, T16>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ktab_tile_kernel<K, EMIT, T16>,
                                                          kKThreads, smem);
        if (e != cudaSuccess) return e;
        per_sm.store(n > 0 ? n : 1);
    }
    *per_sm_out = per_sm.load();
    return cudaSuccess;
}

template <int K, bool EMIT, bool T16>
cudaError_t launch_ktab_k(int sm_count, long long max_tiles, const uint8_t *sym,
                          const long long *srec, const long long *wpre, const long long *tot,
                          const int *klut, const uint16_t *klut16, KtabIds base, long long *tsum,
                          int *out, long long cap, long long *id_offsets, const unsigned *gate,
                          unsigned gate_epoch, cudaStream_t s) {
    constexpr int smem = ktab_smem(K, EMIT, T16);
    int per_sm = 1;
    cudaError_t e = ktab_init<K, EMIT, T16>(&per_sm);
    if (e != cudaSuccess) return e;
    if (!sym) return cudaSuccess;  // (initialization only)
    long long grid = (long long)sm_count * per_sm;
    if (grid > max_tiles) grid = max_tiles;
    if (grid < 1) grid = 1;
    ktab_tile_kernel<K, EMIT, T16><<<(unsigned)grid, kKThreads, smem, s>>>(
        sym, srec, wpre, tot, klut, klut16, base, tsum, out, cap, id_offsets, gate, gate_epoch);
    return cudaGetLastError();
}

cudaError_t launch_ktab(int k, bool emit, bool t16, int sm_count, long long max_tiles,
                        const uint8_t *sym, const long long *srec, const long long *wpre,
                        const long long *tot, const int *klut, const uint16_t *klut16,
                        KtabIds base, long long *tsum, int *out, long long cap,
                        long long *id_offsets, const unsigned *gate, unsigned gate_epoch,
                        cudaStream_t s) {
#define DNATOK_KT(KK, EM, TT)                                                                  \
    return launch_ktab_k<KK, EM, TT>(sm_count, max_tiles, sym, srec, wpre, tot, klut, klut16,  \
                                     base, tsum, out, cap, id_offsets, gate, gate_epoch, s)
#define DNATOK_KT_K(KK)                                                                        \
    case KK:                                                                                   \
        if (emit) {                                                                            \
            if (t16 && KK <= 6) DNATOK_KT(KK, true, (KK <= 6));                                \
            DNATOK_KT(KK, true, false);                                                        \
        } else {                                                                               \
            if (t16 && KK <= 6) DNATOK_KT(KK, false, (KK <= 6));                               \
            DNATOK_KT(KK, false, false);                                                       \
        }
    switch (k) {
        DNATOK_KT_K(1) DNATOK_KT_K(2) DNATOK_KT_K(3) DNATOK_KT_K(4) DNATOK_KT_K(5)
        DNATOK_KT_K(6) DNATOK_KT_K(7) DNATOK_KT_K(8) DNATOK_KT_K(9) DNATOK_KT_K(10)
        default: return cudaErrorInvalidValue;
    }
#undef DNATOK_KT_K
#undef DNATOK_KT
}

void free_ovl(OvlState *o) {
    cudaFree(o->d_sym);
    cudaFree(o->d_srec);
    cudaFree(o->d_wpre);
    cudaFree(o->d_tot);
    cudaFree(o->d_tsum);
    cudaFree(o->d_trec);
    cudaFree(o->d_went);
    o->d_trec = nullptr;
    o->d_went = nullptr;
    o->d_sym = nullptr;
    o->d_srec = nullptr;
    o->d_wpre = nullptr;
    o->d_tot = nullptr;
    o->d_tsum = nullptr;
    o->cap_sym = o->cap_srec = o->cap_tsum = 0;
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
    if (h->mode == DNATOK_KMER_TABLE) {
        // launch limits of the table kernels (a no-op after the first time)
        KtabIds none{};
        for (int emit = 0; emit < 2; ++emit) {
            cudaError_t e = launch_ktab(h->k, emit != 0, h->d_klut16 != nullptr, 1, 1, nullptr,
                                        nullptr, nullptr, nullptr, nullptr, nullptr, none, nullptr,
                                        nullptr, 0, nullptr, nullptr, 0u, s);
            if (e != cudaSuccess) return fail_cuda(h, e, "table k-mer kernel setup");
        }
        if (h->fmt == DNATOK_RAW) {
            cudaError_t e = ktab_direct_setup(h);
            if (e != cudaSuccess) return fail_cuda(h, e, "table k-mer kernel setup (RAW bytes)");
        }
    }
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
    const long long ct = cs_ / kKW + 2;  // tiles of windows (at most one window per symbol)
    e = cudaMalloc(&o->d_sym, (size_t)cs_ + 16);
    if (e == cudaSuccess) e = cudaMalloc(&o->d_srec, sizeof(long long) * (size_t)(cr + 1));
    if (e == cudaSuccess && h->mode == DNATOK_KMER_TABLE)
        e = cudaMalloc(&o->d_wpre, sizeof(long long) * (size_t)(cr + 1));
    if (e == cudaSuccess && h->mode == DNATOK_KMER_TABLE)
        e = cudaMalloc(&o->d_tsum, sizeof(long long) * (size_t)ct);
    if (e == cudaSuccess && h->mode == DNATOK_KMER_TABLE && h->fmt == DNATOK_RAW) {
        const long long nt = ktab_direct_tiles(cs_);
        e = cudaMalloc(&o->d_trec, sizeof(long long) * (size_t)nt);
        if (e == cudaSuccess)
            e = cudaMalloc(&o->d_went, (h->kent16 ? 2 : 4) * (size_t)ktab_direct_entries(cs_, cr, h->k));
    }
    if (e == cudaSuccess) e = cudaMalloc(&o->d_tot, 2 * sizeof(long long));
    if (e != cudaSuccess) {
        free_ovl(o);
        return fail_cuda(h, e, "cudaMalloc(overlapping k-mer workspace)");
    }
    o->cap_sym = cs_;
    o->cap_srec = cr;
    o->cap_tsum = h->mode == DNATOK_KMER_TABLE ? ct : 0;
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
    offsets_kernel<kOffsetsTokens><<<1, kOPlanThreads, 0, s>>>(
        reinterpret_cast<long long *>(id_offsets_d), o->d_srec, nullptr, o->d_tot, h->k,
        offsets_capacity, reinterpret_cast<long long *>(totals_d), h->d_status, nullptr, 0u);
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

__global__ void __launch_bounds__(kTileScanThreads) tile_scan_kernel(
    long long *tsum, const long long *tinv, const long long *keys, const long long *n_rec_dev,
    long long n_rec_host, const long long *n_items_dev, long long n_items_host, int items_per_tile,
    long long *rec_out, long long *totals_out, const int *status, const unsigned *gate,
    unsigned gate_epoch, bool run_if_raised) {
    constexpr int kPer = 4;
    __shared__ long long wsum[kTileScanThreads / 32], winv[kTileScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (dev_failed(status)) return;  // an earlier pass failed: its counts are not valid
    if (gate) {
        // behind a direct path (run_if_raised: only when it declined), or
        // the direct path's own scan (only when it did not)
        const bool raised = *(volatile const unsigned *)gate == gate_epoch;
        if (raised != run_if_raised) return;
    }
    const long long n_rec = n_rec_dev ? *n_rec_dev : n_rec_host;
    if (n_rec < 0) return;
    const long long n_items = n_items_dev ? *n_items_dev : (n_items_host >= 0 ? n_items_host : keys[n_rec]);
    if (n_items < 0) return;
    const long long n_tiles = (n_items + items_per_tile - 1) / items_per_tile;
    long long carry = 0, inv = 0;
    for (long long b0 = 0; b0 < n_tiles; b0 += (long long)kTileScanThreads * kPer) {
        long long v[kPer], sum = 0, isum = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const long long i = b0 + (long long)tid * kPer + j;
            v[j] = i < n_tiles ? tsum[i] : 0;
            if (tinv && i < n_tiles) isum += tinv[i];
            sum += v[j];
        }
        long long x = sum, y = isum;
        for (int o = 1; o < 32; o <<= 1) {
            const long long a = __shfl_up_sync(0xffffffffu, x, o);
            const long long c = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) {
                x += a;
                y += c;
            }
        }
        if (lane == 31) {
            wsum[warp] = x;
            winv[warp] = y;
        }
        __syncthreads();
        long long pre = carry, tt = 0, ti = 0;
        for (int w = 0; w < kTileScanThreads / 32; ++w) {
            if (w < warp) pre += wsum[w];
            tt += wsum[w];
            ti += winv[w];
        }
        long long run = pre + x - sum;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const long long i = b0 + (long long)tid * kPer + j;
            if (i < n_tiles) tsum[i] = run;
            run += v[j];
        }
        carry += tt;
        inv += ti;
        __syncthreads();  // wsum is rewritten by the next pass
    }
    // records with no item left start at the total: the first r with
    // keys[r] >= n_items, then every later one
    long long lo = 0, hi = n_rec;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (keys[mid] >= n_items) hi = mid; else lo = mid + 1;
    }
    for (long long r = lo + tid; r <= n_rec; r += kTileScanThreads) rec_out[r] = carry;
    if (tid == 0 && totals_out) {
        totals_out[0] = carry;
        totals_out[1] = tinv ? inv : n_rec;
    }
}

dnatok_status ktab_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                          const int64_t *seq_offsets_d, int64_t n_seq, int32_t *ids_out_d,
                          int64_t ids_capacity, int64_t *id_offsets_d, int64_t offsets_capacity,
                          int64_t *totals_d, cudaStream_t s) {
    dnatok_status st = ovl_reserve(h, n_bytes, offsets_capacity, s);
    if (st != DNATOK_OK) return st;
    OvlState *o = h->ovl;
    const bool raw = (h->fmt == DNATOK_RAW);
    long long *offs = reinterpret_cast<long long *>(id_offsets_d);
    const long long *so = reinterpret_cast<const long long *>(seq_offsets_d);
    cudaError_t e = cudaSuccess;
    // 0. RAW input: straight from the bytes (window plan, count, scan,
    // emit), with the general path below gated behind it.  Not under stream
    // capture: a replay would find the gate raised with the epoch baked into
    // the graph.
    unsigned gate_ep = 0;
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(s, &capst) == cudaSuccess &&
                           capst != cudaStreamCaptureStatusNone;
    if (raw && h->direct && n_bytes > 0 && !capturing && o->d_trec &&
        direct_eligible(MODE_SYM, n_seq, h->lut_host)) {
        // the general path's workspace first: growing it clears the gate
        // and restarts the epochs, which must not happen behind the gate
        st = ensure_workspace(h, n_bytes, n_seq + 1, h->shape, s);
        if (st != DNATOK_OK) return st;
        st = next_epoch(h, s, &gate_ep);
        if (st != DNATOK_OK) return st;
        e = ktab_direct_launch(h, bytes_d, n_bytes, so, n_seq, o->d_wpre, o->d_trec, o->d_tsum,
                               o->d_went, ids_out_d, ids_capacity, offs,
                               reinterpret_cast<long long *>(totals_d), gate_ep, s);
        if (e != cudaSuccess) return fail_cuda(h, e, "table k-mer launch (RAW bytes)");
    }
    const unsigned *gate = gate_ep ? h->d_gate : nullptr;
    // 1. symbols and record starts (in symbols)
    st = run_tile_encode(h, MODE_SYM, 1, raw ? BSRC_LIST : BSRC_FASTA, bytes_d, n_bytes,
                         raw ? so : nullptr, raw ? n_seq + 1 : 0, o->d_sym, o->cap_sym, offs,
                         offsets_capacity, o->d_tot, nullptr, nullptr, raw ? 0 : 1, raw ? 0 : 1, s,
                         gate_ep);
    if (st != DNATOK_OK) return st;
    if (gate_ep) h->direct_epoch = gate_ep;
    // 2. window offsets
    offsets_kernel<kOffsetsWindows><<<1, kOPlanThreads, 0, s>>>(
        offs, o->d_srec, o->d_wpre, o->d_tot, h->k, offsets_capacity,
        reinterpret_cast<long long *>(totals_d), h->d_status, gate, gate_ep);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e, "window offsets launch");
    // 3-5. count, scan, emit
    const long long tiles = n_bytes / kKW + 1;
    const bool t16 = h->d_klut16 != nullptr;
    KtabIds base;
    for (int d = 0; d < 5; ++d) base.b[d] = h->base_ids[d];
    e = launch_ktab(h->k, false, t16, h->sm_count, tiles, o->d_sym, o->d_srec, o->d_wpre, o->d_tot,
                    h->d_klut, h->d_klut16, base, o->d_tsum, ids_out_d, ids_capacity, offs, gate,
                    gate_ep, s);
    if (e != cudaSuccess) return fail_cuda(h, e, "table k-mer count launch");
    tile_scan_kernel<<<1, kTileScanThreads, 0, s>>>(o->d_tsum, nullptr, o->d_wpre, o->d_tot + 1, 0,
                                                nullptr, -1, kKW, offs,
                                                reinterpret_cast<long long *>(totals_d),
                                                h->d_status, gate, gate_ep, true);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e, "table k-mer scan launch");
    e = launch_ktab(h->k, true, t16, h->sm_count, tiles, o->d_sym, o->d_srec, o->d_wpre, o->d_tot,
                    h->d_klut, h->d_klut16, base, o->d_tsum, ids_out_d, ids_capacity, offs, gate,
                    gate_ep, s);
    if (e != cudaSuccess) return fail_cuda(h, e, "table k-mer emit launch");
    return DNATOK_OK;
}

}  // namespace dnatok
