// bpe.cu -- BPE merge application on the GPU (C7/C8 semantics: greedy
// lowest-rank, leftmost-first merging inside words; a word is a maximal run
// of bases inside one record; an N-class symbol ends the word and emits
// N_ID = 4 + M).  The paper names BPE among the schemes its systems layer
// serves (Sec. 1.1, Sec. 1.3, Sec. 4.3) but gives no GPU algorithm for it.
//
// Method (each fact is pinned by brute force against the oracle in the tests):
//  * Split: a final token boundary at p splits BPE(w) into BPE(w[:p]) and
//    BPE(w[p:]).
//  * A tokenization equals BPE(w) iff every token is self-encoding
//    (BPE(str t) = [t]) and every adjacent pair (a, b) is compatible
//    (BPE(str a + str b) = [a, b]).
//  * So last(j), the last token of BPE of the word prefix ending at symbol
//    j, is the self-encoding suffix token t compatible with last(j - |t|)
//    (anything at the word start): one left-to-right pass over the symbols
//    with a trie of reversed token strings and a compatibility bitmap.
//    Only |last(j)| (one byte per symbol) is stored.
//  * The choice at j depends only on the previous lmax values, so a pass
//    started mid-word (a segment's halo) agrees with the exact pass once a
//    window of lmax values agrees; segments are computed independently and
//    checked against their left neighbour, and the rare failure is redone
//    exactly, in order.
//  * The tokens are the chain j -> j - |last(j)| from the last symbol.  Each
//    segment maps every possible entry (the first chain element at or below
//    its last symbol: lmax choices) to its exit and token count; the maps
//    almost always collapse to one exit, which makes the entries local.
//    Counts are scanned for the output positions; each segment then writes
//    its ids walking its chain backwards.
//
// Kernels per encode: the symbol pass (tile kernel, MODE_SYM), bpe_dp,
// bpe_sync, bpe_repair, bpe_maps, bpe_entries, three scan kernels,
// bpe_emit, bpe_offsets.
#include <algorithm>
#include <cstring>
#include <vector>

#include "handle.h"
#include "tile_kernel.cuh"

using namespace dnatok;

namespace {

constexpr int kMaxTokLen = 32;      // longest supported self-encoding token (bases)
constexpr unsigned kNoTok = 0xFFFFu;
constexpr unsigned kHashEmpty = 0xFFFFFFFFu;
constexpr int kScanItems = 8;       // per thread in the scan kernels
constexpr int kScanThreads = 256;

struct BpeTables {
    int V;            // 4 + M token ids; N_ID = V
    int lmax;         // longest self-encoding token
    int n_deep;       // deep trie nodes (index 0 = "none")
    // tokens of 1..5 bases: direct tables indexed by the d-mer code (last
    // base in the low bits), at offsets 0, 4, 20, 84, 340 (1364 entries)
    const unsigned short *kmtok;
    // tokens of 6+ bases: the last 6 bases index node6 (4096 entries) -> a
    // node of the trie of reversed strings below depth 6
    const unsigned short *node6;
    const uint2 *child;          // per deep node: 4 x u16 children (0 = none)
    const unsigned short *tok;   // per deep node: token id ending here or kNoTok
    const unsigned *compat;      // V x V bits, row = left token
};

// offset of the d-base table: (4^d - 4) / 3 = 0, 4, 20, 84, 340 for d = 1..5
__host__ __device__ constexpr int km_off(int d) { return ((1 << (2 * d)) - 4) / 3; }
constexpr int kKmTotal = 1364;

struct BpeWork {
    const uint8_t *sym;          // symbols 0..3 bases, 4 N-class
    uint8_t *len;                // |last(j)| per symbol
    uint8_t *halo;               // per segment: halo values of its fresh pass
    uint8_t *flags;              // per segment: 1 = exact start
    uint8_t *map_v;              // per segment x 32 entries: exit offset
    unsigned short *map_c;       // per segment x 32 entries: token count
    uint8_t *const_v;            // per segment: common exit or 0xFF
    unsigned *count;             // per segment: tokens on the true chain
    uint8_t *entry;              // per segment: true entry offset
    long long *base;             // per segment: exclusive prefix of count
    long long *block_sums;
    int *bad;                    // [0] = count, then segment ids
    unsigned *bits;              // per segment: token ends, one bit per symbol
    long long *tot;              // {n_sym, n_rec} from the symbol pass
    long long *rec_off;          // record starts (symbols), rewritten as id offsets
    long long offsets_cap;
    int *out;
    long long out_cap;
    long long *totals_out;       // caller's {n_ids, n_records} or null
    int *status;
    int S, H;                    // segment symbols, halo symbols
    long long max_seg;           // segments the grids cover
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned trie_child(const uint2 *child, unsigned node, unsigned c) {
    const uint2 v = child[node];
    const unsigned w = (c < 2) ? v.x : v.y;
    return (c & 1) ? (w >> 16) : (w & 0xFFFFu);
}

__device__ __forceinline__ bool compat_bit(const unsigned *compat, int V, unsigned a, unsigned b) {
    const unsigned long long bit = (unsigned long long)a * (unsigned)V + b;
    return (__ldg(compat + (bit >> 5)) >> (bit & 31)) & 1u;
}

// Token id of the L symbols ending at e (L <= lmax).
__device__ __forceinline__ unsigned token_at(const BpeTables &T, const uint8_t *sym, long long e,
                                             int L) {
    unsigned code = 0;
    const int d0 = L < 6 ? L : 6;
    for (int d = d0; d >= 1; --d) code = (code << 2) | sym[e - d + 1];
    if (L <= 5) return T.kmtok[km_off(L) + code];
    unsigned node = T.node6[code];
    for (int d = 7; d <= L; ++d) node = trie_child(T.child, node, sym[e - d + 1]);
    return T.tok[node];
}

// Largest r with rec_off[r] <= x (rec_off[0] = 0, non-decreasing, n entries).
__device__ __forceinline__ long long rec_upper(const long long *rec_off, long long n, long long x) {
    long long lo = 0, hi = n - 1;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (rec_off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One step of the prefix DP at symbol j (a base).  reg: codes of the word so
// far (newest in the low bits); wd: symbols of the word through j; ring:
// last token ids by position mod 32.  Candidates are tried longest first;
// the first that starts the word or is compatible with the token before it
// is last(j).  Returns (length << 16) | token.
__device__ __forceinline__ unsigned dp_step(const BpeTables &T, unsigned long long reg, int wd,
                                            long long j, const unsigned short *ring) {
    const int dm = wd < T.lmax ? wd : T.lmax;
    auto fits = [&](int d, unsigned t) -> bool {
        if (d == wd) return true;
        return compat_bit(T.compat, T.V, ring[(j - d) & 31], t);
    };
    if (dm >= 6) {
        const unsigned n6 = T.node6[(unsigned)reg & 0xFFFu];
        if (n6) {
            unsigned short deep[kMaxTokLen];
            int nd = 0;
            unsigned node = n6;
            for (int d = 7; d <= dm; ++d) {
                node = trie_child(T.child, node, (unsigned)(reg >> (2 * (d - 1))) & 3u);
                if (!node) break;
                const unsigned t = T.tok[node];
                deep[d - 7] = (unsigned short)t;
                nd = d - 6;
            }
            for (int q = nd - 1; q >= 0; --q) {
                const unsigned t = deep[q];
                if (t != kNoTok && fits(q + 7, t)) return ((unsigned)(q + 7) << 16) | t;
            }
            const unsigned t6 = T.tok[n6];
            if (t6 != kNoTok && fits(6, t6)) return (6u << 16) | t6;
        }
    }
    unsigned t5[5];
#pragma unroll
    for (int d = 1; d <= 5; ++d)
        t5[d - 1] = T.kmtok[km_off(d) + ((unsigned)reg & ((1u << (2 * d)) - 1u))];
#pragma unroll
    for (int d = 5; d >= 2; --d)
        if (d <= dm && t5[d - 1] != kNoTok && fits(d, t5[d - 1])) return ((unsigned)d << 16) | t5[d - 1];
    return (1u << 16) | t5[0];  // a single base: no other candidate fits
}

// ------------------------------------------------------- table building

struct RankHash {
    const unsigned *keys;  // (left << 16) | right, kHashEmpty = free
    const unsigned *vals;  // rank
    unsigned mask;
};

__device__ __forceinline__ unsigned hash_slot(unsigned key) { return (key * 2654435761u) >> 7; }

__device__ __forceinline__ unsigned rank_of(const RankHash &h, unsigned a, unsigned b) {
    const unsigned key = (a << 16) | b;
    unsigned s = hash_slot(key) & h.mask;
    while (true) {
        const unsigned k = h.keys[s];
        if (k == key) return h.vals[s];
        if (k == kHashEmpty) return 0xFFFFFFFFu;
        s = (s + 1) & h.mask;
    }
}

// Greedy BPE (C7) of a short symbol string s[0..n) in place.  boundary >= 0:
// stop and return -1 as soon as a merge would join s[boundary-1] and
// s[boundary] (the crossing that makes a pair incompatible).
__device__ int greedy_bpe(const RankHash &h, unsigned short *s, int n, int boundary) {
    unsigned r[2 * kMaxTokLen];
    for (int i = 0; i + 1 < n; ++i) r[i] = rank_of(h, s[i], s[i + 1]);
    while (n > 1) {
        unsigned best = 0xFFFFFFFFu;
        int bi = -1;
        for (int i = 0; i + 1 < n; ++i)
            if (r[i] < best) {
                best = r[i];
                bi = i;
            }
        if (bi < 0) break;
        if (boundary >= 0 && bi == boundary - 1) return -1;
        s[bi] = (unsigned short)(4 + best);
        for (int i = bi + 1; i + 1 < n; ++i) s[i] = s[i + 1];
        for (int i = bi + 1; i + 2 < n; ++i) r[i] = r[i + 1];
        --n;
        if (bi > 0) r[bi - 1] = rank_of(h, s[bi - 1], s[bi]);
        if (bi + 1 < n) r[bi] = rank_of(h, s[bi], s[bi + 1]);
        if (boundary >= 0 && bi < boundary) --boundary;
    }
    return n;
}

__global__ void bpe_selfenc_kernel(RankHash h, const uint8_t *pool, const int *pool_off,
                                   const int *tok_len, int V, uint8_t *selfenc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= V) return;
    const int L = tok_len[t];
    if (L > kMaxTokLen) {
        selfenc[t] = 0;
        return;
    }
    unsigned short s[2 * kMaxTokLen];
    for (int i = 0; i < L; ++i) s[i] = pool[pool_off[t] + i];
    const int n = greedy_bpe(h, s, L, -1);
    selfenc[t] = (n == 1 && s[0] == t) ? 1 : 0;
}

// One thread per (left token a, 32 right tokens): the 32 bits of row a.
__global__ void bpe_compat_kernel(RankHash h, const uint8_t *pool, const int *pool_off,
                                  const int *tok_len, const uint8_t *selfenc, int V,
                                  unsigned *compat) {
    const long long words_per_row = ((long long)V + 31) / 32;
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)V * words_per_row) return;
    const int a = (int)(gid / words_per_row);
    const int w = (int)(gid % words_per_row);
    unsigned bits = 0;
    if (selfenc[a]) {
        const int La = tok_len[a];
        for (int q = 0; q < 32; ++q) {
            const int b = w * 32 + q;
            if (b >= V || !selfenc[b]) continue;
            const int Lb = tok_len[b];
            unsigned short s[2 * kMaxTokLen];
            for (int i = 0; i < La; ++i) s[i] = pool[pool_off[a] + i];
            for (int i = 0; i < Lb; ++i) s[La + i] = pool[pool_off[b] + i];
            const int n = greedy_bpe(h, s, La + Lb, La);
            if (n == 2) bits |= 1u << q;
        }
    }
    const unsigned long long bit0 = (unsigned long long)a * (unsigned)V + (unsigned)w * 32u;
    // rows are not word-aligned: deposit the 32 bits at their global position
    unsigned *p = compat + (bit0 >> 5);
    const unsigned sh = (unsigned)(bit0 & 31);
    if (bits) {
        atomicOr(p, bits << sh);
        if (sh) atomicOr(p + 1, bits >> (32 - sh));
    }
}

// -------------------------------------------------------- encode kernels

extern __shared__ __align__(16) unsigned char bpe_smem[];

// Copy the lookup tables into shared memory (when they fit) and return the
// tables the block uses.
__device__ BpeTables stage_tables(const BpeTables &G, bool smem) {
    if (!smem) return G;
    uint2 *c = reinterpret_cast<uint2 *>(bpe_smem);
    unsigned short *t = reinterpret_cast<unsigned short *>(c + G.n_deep);
    unsigned short *n6 = t + G.n_deep;
    unsigned short *km = n6 + 4096;
    for (int i = threadIdx.x; i < G.n_deep; i += blockDim.x) {
        c[i] = G.child[i];
        t[i] = G.tok[i];
    }
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) n6[i] = G.node6[i];
    for (int i = threadIdx.x; i < kKmTotal; i += blockDim.x) km[i] = G.kmtok[i];
    __syncthreads();
    BpeTables T = G;
    T.child = c;
    T.tok = t;
    T.node6 = n6;
    T.kmtok = km;
    return T;
}

// The prefix DP over one segment (thread per segment), started lmax..H
// symbols before it unless a word starts closer.
__global__ void __launch_bounds__(256) bpe_dp_kernel(BpeTables G, bool smem, BpeWork W) {
    const BpeTables T = stage_tables(G, smem);
    const long long seg = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0], n_rec = W.tot[1];
    if (n_rec + 1 > W.offsets_cap) {
        if (seg == 0) set_dev_status(W.status, DEV_CAPACITY);
        return;
    }
    const long long s = seg * W.S;
    if (s >= n_sym) return;
    const long long e = (s + W.S < n_sym) ? s + W.S : n_sym;
    const long long nb = n_rec + 1;
    long long r = rec_upper(W.rec_off, nb, s);
    long long a = s - W.H;
    bool exact = false;
    if (a <= W.rec_off[r]) {
        a = W.rec_off[r];
        exact = true;
    }
    while (r + 1 < nb && W.rec_off[r + 1] <= a) ++r;  // empty records at a
    long long next_b = (r + 1 < nb) ? W.rec_off[r + 1] : (1ll << 62);
    unsigned short ring[32];
    unsigned long long reg = 0;
    int wd = 0;
    uint8_t *halo = W.halo + seg * (long long)W.H;
    const long long h0 = s - W.H;  // first halo position (a multiple of 16)
    // 16 symbols per load and 16 lengths per store: s, H and the buffers are
    // 16-byte aligned; a record start inside the halo only shifts where the
    // pass begins within its 16-symbol block
    for (long long j0 = (a > h0 ? a : h0) & ~15ll; j0 < e; j0 += 16) {
        const uint4 sv = *reinterpret_cast<const uint4 *>(W.sym + j0);
        const unsigned long long s_lo = ((unsigned long long)sv.y << 32) | sv.x;
        const unsigned long long s_hi = ((unsigned long long)sv.w << 32) | sv.z;
        unsigned long long l_lo = 0, l_hi = 0;
        const int q0 = (j0 < a) ? (int)(a - j0) : 0;
        const int q1 = (e - j0 < 16) ? (int)(e - j0) : 16;
#pragma unroll 1
        for (int q = q0; q < q1; ++q) {
            const long long j = j0 + q;
            while (j == next_b) {
                wd = 0;
                reg = 0;
                ++r;
                next_b = (r + 1 < nb) ? W.rec_off[r + 1] : (1ll << 62);
            }
            const unsigned c = (unsigned)((q < 8 ? s_lo >> (8 * q) : s_hi >> (8 * (q - 8))) & 0xFFu);
            unsigned L, t;
            if (c >= 4) {
                L = 1;
                t = (unsigned)T.V;
                wd = 0;
                reg = 0;
                if (j < s) exact = true;  // a word starts after it, before the segment
            } else {
                reg = (reg << 2) | c;
                if (wd < 63) ++wd;
                const unsigned pk = dp_step(T, reg, wd, j, ring);
                L = pk >> 16;
                t = pk & 0xFFFFu;
            }
            ring[j & 31] = (unsigned short)t;
            if (q < 8) l_lo |= (unsigned long long)L << (8 * q);
            else l_hi |= (unsigned long long)L << (8 * (q - 8));
        }
        const uint4 lv = make_uint4((unsigned)l_lo, (unsigned)(l_lo >> 32), (unsigned)l_hi,
                                    (unsigned)(l_hi >> 32));
        if (j0 >= s) *reinterpret_cast<uint4 *>(W.len + j0) = lv;
        else if (W.H > 0) *reinterpret_cast<uint4 *>(halo + (j0 - h0)) = lv;
    }
    if (a > h0) {
        // halo positions before the pass began hold 0 (no value)
        for (long long x = h0; x < (a & ~15ll); ++x) halo[x - h0] = 0;
    }
    W.flags[seg] = exact ? 1 : 0;
}

// A segment whose pass did not start exactly is correct if its halo agrees
// with its left neighbour's values over lmax consecutive symbols.
__global__ void bpe_sync_kernel(BpeTables G, BpeWork W) {
    const long long seg = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0];
    const long long s = seg * W.S;
    if (seg == 0 || s >= n_sym || W.flags[seg]) return;
    const uint8_t *halo = W.halo + seg * (long long)W.H;
    int run = 0;
    for (long long j = s - W.H; j < s; ++j) {
        const uint8_t v = halo[j - (s - W.H)];
        run = (v != 0 && v == W.len[j]) ? run + 1 : 0;
        if (run >= G.lmax) return;
    }
    const int q = atomicAdd(W.bad, 1);
    W.bad[1 + q] = (int)seg;
}

// Exact recomputation, in order, of the segments that did not sync (rare):
// rebuild the DP state at the segment start from the (correct) values to its
// left, recompute the whole segment, then re-check the next one against the
// new values and continue into it if it no longer syncs.
__global__ void bpe_repair_kernel(BpeTables T, BpeWork W) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (dev_failed(W.status)) return;
    const int nbad = W.bad[0];
    if (nbad == 0) return;
    int *list = W.bad + 1;
    for (int i = 1; i < nbad; ++i) {  // insertion sort (short list)
        const int v = list[i];
        int k = i - 1;
        while (k >= 0 && list[k] > v) {
            list[k + 1] = list[k];
            --k;
        }
        list[k + 1] = v;
    }
    const long long n_sym = W.tot[0], nb = W.tot[1] + 1;
    long long done_until = 0;  // symbols below this are final
    for (int i = 0; i < nbad; ++i) {
        long long seg = list[i];
        long long s = seg * W.S;
        if (s < done_until) continue;
        // DP state at s from the values to its left
        unsigned short ring[32];
        unsigned long long reg = 0;
        int wd = 0;
        long long r = rec_upper(W.rec_off, nb, s);
        while (r + 1 < nb && W.rec_off[r + 1] <= s) ++r;
        const long long ws = W.rec_off[r];
        long long x = s - 1;
        while (x >= ws && x >= s - 63 && W.sym[x] < 4) --x;
        // symbols (x, s) are the word so far (capped at 63)
        for (long long y = x + 1; y < s; ++y) {
            reg = (reg << 2) | W.sym[y];
            ++wd;
        }
        for (long long y = (s - 32 > 0 ? s - 32 : 0); y < s; ++y)
            ring[y & 31] = (W.sym[y] >= 4) ? (unsigned short)T.V
                                           : (unsigned short)token_at(T, W.sym, y, W.len[y]);
        long long next_b = (r + 1 < nb) ? W.rec_off[r + 1] : (1ll << 62);
        while (true) {
            const long long e = (s + W.S < n_sym) ? s + W.S : n_sym;
            for (long long j = s; j < e; ++j) {
                while (j == next_b) {
                    wd = 0;
                    reg = 0;
                    ++r;
                    next_b = (r + 1 < nb) ? W.rec_off[r + 1] : (1ll << 62);
                }
                const unsigned c = W.sym[j];
                unsigned L, t;
                if (c >= 4) {
                    L = 1;
                    t = (unsigned)T.V;
                    wd = 0;
                    reg = 0;
                } else {
                    reg = (reg << 2) | c;
                    if (wd < 63) ++wd;
                    const unsigned pk = dp_step(T, reg, wd, j, ring);
                    L = pk >> 16;
                    t = pk & 0xFFFFu;
                }
                ring[j & 31] = (unsigned short)t;
                W.len[j] = (uint8_t)L;
            }
            done_until = e;
            ++seg;
            s = seg * W.S;
            if (s >= n_sym || W.flags[seg]) break;
            // does the next segment's fresh pass agree with the new values?
            const uint8_t *halo = W.halo + seg * (long long)W.H;
            int run = 0;
            bool ok = false;
            for (long long j = s - W.H; j < s && !ok; ++j) {
                const uint8_t v = halo[j - (s - W.H)];
                run = (v != 0 && v == W.len[j]) ? run + 1 : 0;
                ok = run >= T.lmax;
            }
            if (ok) break;
        }
    }
}

// Warp per segment, lane u = entry offset: walk the chain from symbol
// end - 1 - u down past the segment start.
__global__ void bpe_maps_kernel(BpeTables G, BpeWork W) {
    const long long seg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int u = threadIdx.x & 31;
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0];
    const long long s = seg * W.S;
    if (s >= n_sym) return;
    const long long e_end = (s + W.S < n_sym) ? s + W.S : n_sym;
    long long e = e_end - 1 - u;
    unsigned cnt = 0;
    if (u < G.lmax) {
        while (e >= s) {
            e -= W.len[e];
            ++cnt;
        }
    }
    const unsigned v = (unsigned)(s - 1 - e);
    W.map_v[seg * 32 + u] = (uint8_t)v;
    W.map_c[seg * 32 + u] = (unsigned short)cnt;
    const unsigned mine = (u < G.lmax) ? v : 0xFFFFFFFFu;
    const unsigned first = __shfl_sync(0xffffffffu, v, 0);
    const bool same = __all_sync(0xffffffffu, mine == 0xFFFFFFFFu || mine == first);
    if (u == 0) W.const_v[seg] = same ? (uint8_t)first : (uint8_t)0xFF;
}

// The true entry of every segment: the exit of its right neighbour, found
// locally when that neighbour's map is constant (the usual case).
__global__ void bpe_entries_kernel(BpeTables G, BpeWork W) {
    const long long seg = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0];
    const long long n_seg = (n_sym + W.S - 1) / W.S;
    if (seg >= n_seg) {
        if (seg < W.max_seg) W.count[seg] = 0;
        return;
    }
    unsigned u = 0;
    if (seg < n_seg - 1) {
        long long k = seg + 1;
        while (k < n_seg - 1 && W.const_v[k] == 0xFF) ++k;
        u = (W.const_v[k] != 0xFF) ? W.const_v[k] : W.map_v[k * 32 + 0];
        for (long long q = k - 1; q > seg; --q) u = W.map_v[q * 32 + u];
    }
    W.entry[seg] = (uint8_t)u;
    W.count[seg] = W.map_c[seg * 32 + u];
}

// Exclusive scan of the per-segment counts: block sums, one block over the
// block sums, then per-block rescan.
__device__ __forceinline__ long long block_excl_scan(long long v, long long *total) {
    __shared__ long long warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    long long off = 0, all = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < warp) off += warp_tot[w];
        all += warp_tot[w];
    }
    __syncthreads();
    *total = all;
    return off + x - v;
}

__global__ void __launch_bounds__(kScanThreads) bpe_scan_reduce(BpeWork W) {
    const long long i0 = (blockIdx.x * (long long)kScanThreads + threadIdx.x) * kScanItems;
    long long sum = 0;
    for (int q = 0; q < kScanItems; ++q)
        if (i0 + q < W.max_seg) sum += W.count[i0 + q];
    long long total;
    block_excl_scan(sum, &total);
    if (threadIdx.x == 0) W.block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) bpe_scan_top(BpeWork W, long long n_blocks) {
    long long carry = 0;
    for (long long b0 = 0; b0 < n_blocks; b0 += kScanThreads) {
        const long long b = b0 + threadIdx.x;
        const long long v = (b < n_blocks) ? W.block_sums[b] : 0;
        long long total;
        const long long ex = block_excl_scan(v, &total);
        if (b < n_blocks) W.block_sums[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        W.base[W.max_seg] = carry;
        if (!dev_failed(W.status) && W.totals_out) {
            W.totals_out[0] = carry;
            W.totals_out[1] = W.tot[1];
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) bpe_scan_down(BpeWork W) {
    const long long i0 = (blockIdx.x * (long long)kScanThreads + threadIdx.x) * kScanItems;
    long long sum = 0;
    for (int q = 0; q < kScanItems; ++q)
        if (i0 + q < W.max_seg) sum += W.count[i0 + q];
    long long total;
    long long run = W.block_sums[blockIdx.x] + block_excl_scan(sum, &total);
    for (int q = 0; q < kScanItems; ++q)
        if (i0 + q < W.max_seg) {
            W.base[i0 + q] = run;
            run += W.count[i0 + q];
        }
}

// Thread per segment walks its chain (from its entry, backwards) and marks
// the token ends in a bitmap, one bit per symbol, in global memory; then each
// warp emits its 32 segments one after another with lane w taking bitmap word
// w (symbols 32w..32w+31), so the warp writes one contiguous run of ids.
__global__ void __launch_bounds__(256) bpe_emit_kernel(BpeTables G, bool smem, BpeWork W) {
    const BpeTables T = stage_tables(G, smem);
    const int lane = threadIdx.x & 31;
    const long long seg = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0];
    const long long n_seg = (n_sym + W.S - 1) / W.S;
    const int words = (W.S + 31) / 32;
    if (seg < n_seg) {
        const long long s = seg * W.S;
        const long long e_end = (s + W.S < n_sym) ? s + W.S : n_sym;
        unsigned *bits = W.bits + seg * words;
        long long e = e_end - 1 - W.entry[seg];
        int cw = words - 1;
        unsigned acc = 0;
        while (e >= s) {
            const int x = (int)(e - s);
            while ((x >> 5) < cw) {
                bits[cw--] = acc;
                acc = 0;
            }
            acc |= 1u << (x & 31);
            e -= W.len[e];
        }
        for (; cw >= 0; --cw) {
            bits[cw] = acc;
            acc = 0;
        }
    }
    __syncwarp();
    const long long seg0 = seg - lane;
    for (int i = 0; i < 32; ++i) {
        const long long sg = seg0 + i;
        if (sg >= n_seg) break;
        const long long s = sg * W.S;
        const unsigned *bits = W.bits + sg * words;
        long long out = W.base[sg];
        for (int w0 = 0; w0 < words; w0 += 32) {
            const int w = w0 + lane;
            const unsigned wb = (w < words) ? bits[w] : 0u;
            const unsigned c = __popc(wb);
            unsigned x = c;  // inclusive scan of the counts over the warp
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            long long pos = out + (x - c);
            unsigned m = wb;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const long long j = s + 32ll * w + b;
                const unsigned id = (W.sym[j] >= 4) ? (unsigned)T.V : token_at(T, W.sym, j, W.len[j]);
                if (pos >= 0 && pos < W.out_cap) W.out[pos] = (int)id;
                ++pos;
            }
            out += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

// Record starts (in symbols) -> record starts (in ids), in place.
__global__ void bpe_offsets_kernel(BpeWork W) {
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0], nb = W.tot[1] + 1;
    const long long total = W.base[W.max_seg];
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nb;
         r += (long long)gridDim.x * blockDim.x) {
        const long long rho = W.rec_off[r];
        long long off;
        if (rho >= n_sym) {
            off = total;
        } else {
            const long long seg = rho / W.S, s = seg * W.S;
            off = W.base[seg];
            long long e = rho - 1, c = 0;
            while (e >= s) {
                e -= W.len[e];
                ++c;
            }
            off += c;
        }
        W.rec_off[r] = off;
    }
}

}  // namespace

// ======================================================================= host

struct BpeState {
    int M = 0, V = 0, lmax = 1, n_nodes = 1;  // n_nodes: deep trie nodes
    uint2 *d_child = nullptr;
    unsigned short *d_tok = nullptr;
    unsigned short *d_node6 = nullptr;
    unsigned short *d_kmtok = nullptr;
    unsigned *d_compat = nullptr;
    int S = 1024, H = 64;

    // workspace
    long long cap_bytes = -1;
    uint8_t *d_sym = nullptr, *d_len = nullptr, *d_halo = nullptr, *d_flags = nullptr;
    uint8_t *d_map_v = nullptr, *d_const = nullptr, *d_entry = nullptr;
    unsigned short *d_map_c = nullptr;
    unsigned *d_count = nullptr;
    long long *d_base = nullptr, *d_bsums = nullptr, *d_tot = nullptr;
    int *d_bad = nullptr;
    unsigned *d_bits = nullptr;
    long long seg_cap = 0;
    int ws_S = 0, ws_H = 0;
};

namespace {

void free_workspace(BpeState *b) {
    cudaFree(b->d_sym);
    cudaFree(b->d_len);
    cudaFree(b->d_halo);
    cudaFree(b->d_flags);
    cudaFree(b->d_map_v);
    cudaFree(b->d_const);
    cudaFree(b->d_entry);
    cudaFree(b->d_map_c);
    cudaFree(b->d_count);
    cudaFree(b->d_base);
    cudaFree(b->d_bsums);
    cudaFree(b->d_tot);
    cudaFree(b->d_bad);
    cudaFree(b->d_bits);
    b->d_bits = nullptr;
    b->d_sym = b->d_len = b->d_halo = b->d_flags = b->d_map_v = b->d_const = b->d_entry = nullptr;
    b->d_map_c = nullptr;
    b->d_count = nullptr;
    b->d_base = b->d_bsums = b->d_tot = nullptr;
    b->d_bad = nullptr;
    b->cap_bytes = -1;
    b->seg_cap = 0;
}

long long scan_blocks(long long n) {
    const long long per = (long long)kScanThreads * kScanItems;
    return (n + per - 1) / per;
}

dnatok_status ensure_bpe_workspace(dnatok_handle *h, long long n_bytes, cudaStream_t s) {
    BpeState *b = h->bpe;
    if (n_bytes <= b->cap_bytes && b->ws_S == b->S && b->ws_H == b->H) return DNATOK_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(h, DNATOK_ERR_STATE,
                    "BPE workspace must grow during stream capture; call dnatok_reserve first");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaDeviceSynchronize");
    free_workspace(b);
    const long long cap = n_bytes + n_bytes / 8 + 4096;
    const long long nseg = (cap + b->S - 1) / b->S + 1;
    const long long nblk = scan_blocks(nseg) + 1;
    size_t sz[] = {(size_t)cap + 16, (size_t)cap + 16, (size_t)(nseg * b->H + 16), (size_t)nseg,
                   (size_t)nseg * 32, (size_t)nseg, (size_t)nseg, (size_t)nseg * 32 * 2,
                   (size_t)nseg * 4, (size_t)(nseg + 1) * 8, (size_t)nblk * 8, 16,
                   (size_t)(nseg + 1) * 4, (size_t)nseg * 4 * ((b->S + 31) / 32) + 16};
    void **ptr[] = {(void **)&b->d_sym,   (void **)&b->d_len,   (void **)&b->d_halo,
                    (void **)&b->d_flags, (void **)&b->d_map_v, (void **)&b->d_const,
                    (void **)&b->d_entry, (void **)&b->d_map_c, (void **)&b->d_count,
                    (void **)&b->d_base,  (void **)&b->d_bsums, (void **)&b->d_tot,
                    (void **)&b->d_bad,   (void **)&b->d_bits};
    for (int i = 0; i < 14; ++i) {
        e = cudaMalloc(ptr[i], sz[i]);
        if (e != cudaSuccess) {
            free_workspace(b);
            return fail_cuda(h, e, "cudaMalloc(BPE workspace)");
        }
    }
    b->cap_bytes = cap;
    b->seg_cap = nseg;
    b->ws_S = b->S;
    b->ws_H = b->H;
    return DNATOK_OK;
}

size_t trie_smem_bytes(const BpeState *b) {
    return (size_t)b->n_nodes * (sizeof(uint2) + sizeof(unsigned short)) +
           sizeof(unsigned short) * (4096 + kKmTotal) + 16;
}

}  // namespace

namespace dnatok {

dnatok_status bpe_create(dnatok_handle *h, const int32_t *merges, int32_t n_merges) {
    if (n_merges < 0 || n_merges > DNATOK_MAX_MERGES)
        return fail(h, DNATOK_ERR_TABLE, "n_merges must be in [0, DNATOK_MAX_MERGES]");
    const int M = n_merges, V = 4 + M;
    std::vector<std::pair<int, int>> pairs(M);
    std::vector<unsigned long long> keys(M);
    for (int r = 0; r < M; ++r) {
        const int a = merges[2 * r], c = merges[2 * r + 1];
        if (a < 0 || c < 0 || a >= 4 + r || c >= 4 + r)
            return fail(h, DNATOK_ERR_TABLE, "merge " + std::to_string(r) +
                                                 ": operands must be ids below 4 + rank");
        pairs[r] = {a, c};
        keys[r] = ((unsigned long long)a << 32) | (unsigned)c;
    }
    {
        std::vector<unsigned long long> k2 = keys;
        std::sort(k2.begin(), k2.end());
        if (std::adjacent_find(k2.begin(), k2.end()) != k2.end())
            return fail(h, DNATOK_ERR_TABLE, "duplicate merge pair");
    }
    // token strings (only tokens up to kMaxTokLen bases can be self-encoding
    // candidates; longer ones are rejected below if they would be needed)
    std::vector<int> len(V);
    for (int t = 0; t < 4; ++t) len[t] = 1;
    for (int r = 0; r < M; ++r) {
        const long long l = (long long)len[pairs[r].first] + len[pairs[r].second];
        len[4 + r] = (int)(l > kMaxTokLen + 1 ? kMaxTokLen + 1 : l);
    }
    std::vector<int> pool_off(V);
    std::vector<uint8_t> pool;
    std::vector<std::vector<uint8_t>> str(V);
    for (int t = 0; t < V; ++t) {
        if (t < 4) str[t] = {(uint8_t)t};
        else if (len[t] <= kMaxTokLen) {
            str[t] = str[pairs[t - 4].first];
            str[t].insert(str[t].end(), str[pairs[t - 4].second].begin(),
                          str[pairs[t - 4].second].end());
        }
        pool_off[t] = (int)pool.size();
        pool.insert(pool.end(), str[t].begin(), str[t].end());
    }
    // pair -> rank hash
    unsigned hsize = 1024;
    while (hsize < 2u * (unsigned)M + 16) hsize <<= 1;
    std::vector<unsigned> hk(hsize, kHashEmpty), hv(hsize, 0);
    for (int r = 0; r < M; ++r) {
        const unsigned key = ((unsigned)pairs[r].first << 16) | (unsigned)pairs[r].second;
        unsigned sidx = ((key * 2654435761u) >> 7) & (hsize - 1);
        while (hk[sidx] != kHashEmpty) sidx = (sidx + 1) & (hsize - 1);
        hk[sidx] = key;
        hv[sidx] = (unsigned)r;
    }
    BpeState *b = new (std::nothrow) BpeState();
    if (!b) return fail(h, DNATOK_ERR_NOMEM, "host allocation failed");
    h->bpe = b;
    b->M = M;
    b->V = V;
    unsigned *d_hk = nullptr, *d_hv = nullptr;
    uint8_t *d_pool = nullptr, *d_self = nullptr;
    int *d_off = nullptr, *d_len = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_hk);
        cudaFree(d_hv);
        cudaFree(d_pool);
        cudaFree(d_self);
        cudaFree(d_off);
        cudaFree(d_len);
    };
    cudaError_t e = cudaMalloc(&d_hk, hsize * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_hv, hsize * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_pool, pool.size() + 16);
    if (e == cudaSuccess) e = cudaMalloc(&d_self, V);
    if (e == cudaSuccess) e = cudaMalloc(&d_off, V * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_len, V * 4);
    if (e == cudaSuccess) e = cudaMemcpy(d_hk, hk.data(), hsize * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_hv, hv.data(), hsize * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_pool, pool.data(), pool.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_off, pool_off.data(), V * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_len, len.data(), V * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cleanup();
        return fail_cuda(h, e, "BPE table upload");
    }
    RankHash rh{d_hk, d_hv, hsize - 1};
    bpe_selfenc_kernel<<<(V + 127) / 128, 128>>>(rh, d_pool, d_off, d_len, V, d_self);
    std::vector<uint8_t> self(V);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(self.data(), d_self, V, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cleanup();
        return fail_cuda(h, e, "BPE self-encoding pass");
    }
    for (int t = 0; t < V; ++t)
        if (len[t] > kMaxTokLen) {
            // can such a token ever be emitted?  Only if it is self-encoding;
            // its string is too long to check here, so refuse the table.
            cleanup();
            return fail(h, DNATOK_ERR_TABLE, "BPE tokens longer than 32 bases are not supported");
        }
    // trie over reversed strings of self-encoding tokens
    std::vector<unsigned> ch(4, 0);
    std::vector<unsigned short> tk(1, (unsigned short)kNoTok);
    int lmax = 1;
    for (int t = 0; t < V; ++t) {
        if (!self[t]) continue;
        lmax = std::max(lmax, len[t]);
        unsigned node = 0;
        for (int d = 0; d < len[t]; ++d) {
            const unsigned c = str[t][len[t] - 1 - d];
            if (!ch[node * 4 + c]) {
                ch[node * 4 + c] = (unsigned)tk.size();
                tk.push_back((unsigned short)kNoTok);
                ch.insert(ch.end(), {0, 0, 0, 0});
            }
            node = ch[node * 4 + c];
        }
        tk[node] = (unsigned short)t;
    }
    if (tk.size() > 65535) {
        cleanup();
        return fail(h, DNATOK_ERR_TABLE, "BPE token trie exceeds 65535 nodes");
    }
    // Split the lookup: tokens of 1..5 bases in direct tables by their code
    // (last base in the low bits); the 6-base suffix indexes node6, which
    // points into the part of the trie at depth >= 6 (renumbered from 1).
    std::vector<unsigned short> kmtok(kKmTotal, (unsigned short)kNoTok);
    std::vector<unsigned short> node6(4096, 0);
    std::vector<int> depth(tk.size(), 0), deep_id(tk.size(), 0);
    std::vector<unsigned> code(tk.size(), 0);
    std::vector<unsigned> order(1, 0);  // BFS over the full trie
    int n_deep = 1;                     // deep index 0 = none
    for (size_t qi = 0; qi < order.size(); ++qi) {
        const unsigned u = order[qi];
        if (depth[u] >= 6) deep_id[u] = n_deep++;
        if (depth[u] >= 1 && depth[u] <= 5 && tk[u] != kNoTok) kmtok[km_off(depth[u]) + code[u]] = tk[u];
        for (unsigned c = 0; c < 4; ++c) {
            const unsigned v = ch[u * 4 + c];
            if (!v) continue;
            depth[v] = depth[u] + 1;
            // reversed path: the d-th symbol back from the end lands at bits 2(d-1)
            code[v] = depth[v] <= 6 ? code[u] | (c << (2 * (depth[v] - 1))) : code[u];
            order.push_back(v);
        }
    }
    std::vector<uint2> child(n_deep, make_uint2(0, 0));
    std::vector<unsigned short> dtok(n_deep, (unsigned short)kNoTok);
    for (size_t u = 0; u < tk.size(); ++u) {
        if (depth[u] < 6) continue;
        const int id = deep_id[u];
        if (depth[u] == 6) node6[code[u]] = (unsigned short)id;
        dtok[id] = tk[u];
        unsigned cc[4];
        for (int c = 0; c < 4; ++c) cc[c] = ch[u * 4 + c] ? (unsigned)deep_id[ch[u * 4 + c]] : 0u;
        child[id].x = cc[0] | (cc[1] << 16);
        child[id].y = cc[2] | (cc[3] << 16);
    }
    b->lmax = lmax;
    b->n_nodes = n_deep;
    b->H = std::max(64, ((4 * lmax + 15) / 16) * 16);
    const unsigned long long nbits = (unsigned long long)V * V;
    const size_t cwords = (size_t)((nbits + 31) / 32) + 2;
    e = cudaMalloc(&b->d_child, sizeof(uint2) * n_deep);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tok, sizeof(unsigned short) * n_deep);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_node6, sizeof(unsigned short) * 4096);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_kmtok, sizeof(unsigned short) * kKmTotal);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_compat, cwords * 4);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_child, child.data(), sizeof(uint2) * n_deep, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_tok, dtok.data(), sizeof(unsigned short) * n_deep, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_node6, node6.data(), sizeof(unsigned short) * 4096, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_kmtok, kmtok.data(), sizeof(unsigned short) * kKmTotal,
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_compat, 0, cwords * 4);
    if (e == cudaSuccess) {
        const long long threads = (long long)V * ((V + 31) / 32);
        bpe_compat_kernel<<<(unsigned)((threads + 127) / 128), 128>>>(rh, d_pool, d_off, d_len,
                                                                      d_self, V, b->d_compat);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cleanup();
    if (e != cudaSuccess) return fail_cuda(h, e, "BPE compatibility table");
    return DNATOK_OK;
}

void bpe_destroy(dnatok_handle *h) {
    BpeState *b = h->bpe;
    if (!b) return;
    free_workspace(b);
    cudaFree(b->d_child);
    cudaFree(b->d_tok);
    cudaFree(b->d_node6);
    cudaFree(b->d_kmtok);
    cudaFree(b->d_compat);
    delete b;
    h->bpe = nullptr;
}

dnatok_status bpe_reserve(dnatok_handle *h, long long max_bytes) {
    return ensure_bpe_workspace(h, max_bytes, 0);
}

dnatok_status bpe_set_launch(dnatok_handle *h, int seg_symbols, int halo) {
    BpeState *b = h->bpe;
    if (!b) return fail(h, DNATOK_ERR_STATE, "not a BPE handle");
    if (seg_symbols < 64 || seg_symbols > 65536 || (seg_symbols & 15) || halo < 0 ||
        halo > seg_symbols || (halo & 15) || seg_symbols < 2 * b->lmax)
        return fail(h, DNATOK_ERR_ARG, "bad BPE segment / halo");
    b->S = seg_symbols;
    b->H = halo;
    return DNATOK_OK;
}

dnatok_status bpe_stats(dnatok_handle *h, long long *out, cudaStream_t s) {
    BpeState *b = h->bpe;
    if (!b) return fail(h, DNATOK_ERR_STATE, "not a BPE handle");
    out[0] = out[1] = out[2] = 0;
    if (!b->d_tot || !b->d_bad) return DNATOK_OK;  // nothing encoded yet
    long long tot[2] = {0, 0};
    int bad = 0;
    cudaError_t e = cudaMemcpyAsync(tot, b->d_tot, sizeof(tot), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, b->d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e, "BPE statistics read");
    out[0] = tot[0];
    out[1] = (tot[0] + b->ws_S - 1) / (b->ws_S > 0 ? b->ws_S : 1);
    out[2] = bad;
    return DNATOK_OK;
}

dnatok_status bpe_get_launch(const dnatok_handle *h, int *seg_symbols, int *halo) {
    if (!h->bpe) return DNATOK_ERR_STATE;
    *seg_symbols = h->bpe->S;
    *halo = h->bpe->H;
    return DNATOK_OK;
}

dnatok_status bpe_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                         const int64_t *seq_offsets_d, int64_t n_seq, int32_t *ids_out_d,
                         int64_t ids_capacity, int64_t *id_offsets_d, int64_t offsets_capacity,
                         int64_t *totals_d, cudaStream_t s) {
    BpeState *b = h->bpe;
    dnatok_status st = ensure_bpe_workspace(h, n_bytes, s);
    if (st != DNATOK_OK) return st;
    // 1. symbols and record starts (in symbols) from the tile kernel
    const bool raw = (h->fmt == DNATOK_RAW);
    st = run_tile_encode(h, MODE_SYM, 1, raw ? BSRC_LIST : BSRC_FASTA, bytes_d, n_bytes,
                         reinterpret_cast<const long long *>(seq_offsets_d),
                         raw ? n_seq + 1 : 0, b->d_sym, b->cap_bytes,
                         reinterpret_cast<long long *>(id_offsets_d), offsets_capacity, b->d_tot,
                         nullptr, nullptr, raw ? 0 : 1, raw ? 0 : 1, s);
    if (st != DNATOK_OK) return st;
    cudaError_t e = cudaMemsetAsync(b->d_bad, 0, sizeof(int), s);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemsetAsync");

    BpeTables T{b->V, b->lmax, b->n_nodes, b->d_kmtok, b->d_node6, b->d_child, b->d_tok, b->d_compat};
    BpeWork W;
    std::memset(&W, 0, sizeof(W));
    W.sym = b->d_sym;
    W.len = b->d_len;
    W.halo = b->d_halo;
    W.flags = b->d_flags;
    W.map_v = b->d_map_v;
    W.map_c = b->d_map_c;
    W.const_v = b->d_const;
    W.count = b->d_count;
    W.entry = b->d_entry;
    W.base = b->d_base;
    W.block_sums = b->d_bsums;
    W.bad = b->d_bad;
    W.bits = b->d_bits;
    W.tot = b->d_tot;
    W.rec_off = reinterpret_cast<long long *>(id_offsets_d);
    W.offsets_cap = offsets_capacity;
    W.out = ids_out_d;
    W.out_cap = ids_capacity;
    W.totals_out = reinterpret_cast<long long *>(totals_d);
    W.status = h->d_status;
    W.S = b->S;
    W.H = b->H;
    W.max_seg = (n_bytes + b->S - 1) / b->S;
    if (W.max_seg == 0) W.max_seg = 1;

    const size_t smem = trie_smem_bytes(b);
    const bool use_smem = smem <= 96 * 1024 + 16;
    const size_t dyn = use_smem ? smem : 0;
    static bool attr_done = false;  // once per process: allow the largest trie we stage
    if (!attr_done) {
        cudaFuncSetAttribute(bpe_dp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024 + 16);
        cudaFuncSetAttribute(bpe_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024 + 16);
        attr_done = true;
    }
    const unsigned g128 = (unsigned)((W.max_seg + 127) / 128);
    const unsigned g256 = (unsigned)((W.max_seg + 255) / 256);
    bpe_dp_kernel<<<g256, 256, dyn, s>>>(T, use_smem, W);
    bpe_sync_kernel<<<g128, 128, 0, s>>>(T, W);
    bpe_repair_kernel<<<1, 32, 0, s>>>(T, W);
    bpe_maps_kernel<<<(unsigned)((W.max_seg * 32 + 127) / 128), 128, 0, s>>>(T, W);
    bpe_entries_kernel<<<g128, 128, 0, s>>>(T, W);
    const long long nblk = scan_blocks(W.max_seg);
    bpe_scan_reduce<<<(unsigned)nblk, kScanThreads, 0, s>>>(W);
    bpe_scan_top<<<1, kScanThreads, 0, s>>>(W, nblk);
    bpe_scan_down<<<(unsigned)nblk, kScanThreads, 0, s>>>(W);
    // the emit takes its positions from the scans: launch it only if they launched
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e, "BPE kernel launch");
    bpe_emit_kernel<<<g256, 256, dyn, s>>>(T, use_smem, W);
    const long long nrec_bound = raw ? n_seq + 1 : offsets_capacity;
    long long og = (nrec_bound + 255) / 256;
    if (og > 4096) og = 4096;
    if (og < 1) og = 1;
    bpe_offsets_kernel<<<(unsigned)og, 256, 0, s>>>(W);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e, "BPE kernel launch");
    return DNATOK_OK;
}

}  // namespace dnatok
