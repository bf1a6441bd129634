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
//  * So last(j), the token of BPE of the word prefix ending at symbol j that
//    ends at j, is the longest self-encoding token t ending at j that starts
//    the word or is compatible with last(j - |t|): one left-to-right pass.
//    The candidates at j are the tokens that are suffixes of the text read so
//    far; an Aho-Corasick automaton over the token strings gives them, longest
//    first, from its state (one 16-byte node record per step: the state's
//    four transitions and its first two candidates, and a link to the rest).
//    Compatibility is one bit of a V x V bitmap (L2-resident).
//  * The choice at j depends only on the previous lmax values, so a pass
//    started mid-word (a segment's halo) agrees with the exact pass once a
//    window of lmax values agrees; segments are computed independently and
//    checked against their left neighbour, and the rare failure is redone
//    exactly, in order, within the run of segments that depend on it.
//  * The tokens are the chain j -> j - |last(j)| from the last symbol.  Each
//    segment's pass also carries, for every position, where the chain from
//    there leaves the segment and how many tokens it holds, so the segment's
//    map from each of its lmax possible entries to (exit, count) comes out of
//    the same pass.  The maps almost always collapse to one exit, which makes
//    the entries local.  Counts are scanned for the output positions; each
//    segment then writes its ids walking its chain backwards.
//
// Kernels per encode: the symbol pass (tile kernel, MODE_SYM), bpe_dp,
// bpe_sync, three kernels that list the segments to repair in order with the
// region each belongs to, bpe_repair, bpe_entries, three scan kernels,
// bpe_emit, bpe_offsets.
#include <algorithm>
#include <cstring>
#include <vector>

#include "handle.h"
#include "tile_kernel.cuh"

using namespace dnatok;

namespace {

constexpr int kMaxTokLen = 32;      // longest supported self-encoding token (bases)
constexpr unsigned kNone16 = 0xFFFFu;
constexpr unsigned kHashEmpty = 0xFFFFFFFFu;
constexpr int kScanItems = 8;       // per thread in the scan kernels
constexpr int kScanThreads = 256;
constexpr int kDpThreads = 128;     // threads (segments) per block of the merge pass

// Automaton node record (16 bytes): x, y = transitions on A, C | G, T (u16
// each); z = first two candidate tokens (u16 each, 0xFFFF = none); w =
// their lengths (6 bits each) and, in the top 16 bits, the node whose record
// starts the rest of the candidate list (0xFFFF = none).  Candidates are the
// self-encoding tokens that are suffixes of the node's string, longest first.
struct BpeTables {
    int V;                 // 4 + M token ids; N_ID = V
    int lmax;              // longest self-encoding token
    int n_nodes;           // automaton nodes
    const uint4 *node;     // automaton, node 0 = root (empty string)
    const uint8_t *tok_len;  // V + 1 entries (N_ID has length 1)
    const unsigned *compat;  // V x V bits, row = left token
};

struct BpeWork {
    const uint8_t *sym;          // symbols 0..3 bases, 4 N-class
    unsigned short *tok;         // last(j) per symbol (N_ID for an N-class symbol)
    unsigned short *halo;        // per segment: halo values of its fresh pass (0xFFFF: none)
    uint8_t *flags;              // per segment: 1 = exact start
    uint8_t *bad;                // per segment: 1 = its halo did not agree
    uint8_t *map_v;              // per segment x 32 entries: exit offset
    unsigned *map_c;             // per segment x 32 entries: token count
    uint8_t *const_v;            // per segment: common exit or 0xFF
    unsigned *count;             // per segment: tokens on the true chain
    uint8_t *entry;              // per segment: true entry offset
    long long *base;             // per segment: exclusive prefix of count
    long long *block_sums;
    long long *rep_sums;         // block sums of the repair listing (count, region)
    int *n_bad;                  // segments whose halo did not agree
    int *rep_list;               // segments to repair, in order
    int *rep_region;             // per listed segment: the last exact segment before it
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

// (token ids are below 0xFFFF, so a * V + b fits in 32 bits)
__device__ __forceinline__ bool compat_bit(const unsigned *compat, int V, unsigned a, unsigned b) {
    const unsigned bit = a * (unsigned)V + b;
    return (__ldg(compat + (bit >> 5)) >> (bit & 31)) & 1u;
}

__device__ __forceinline__ unsigned node_next(const uint4 &nd, unsigned c) {
    const unsigned w = (c < 2) ? nd.x : nd.y;
    return (c & 1) ? (w >> 16) : (w & 0xFFFFu);
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

// Node records: from the copy in dynamic shared memory (SM) or from global
// memory through the read-only cache.
extern __shared__ __align__(16) uint4 bpe_dyn[];
template <bool SM>
__device__ __forceinline__ uint4 node_at(const BpeTables &T, unsigned i) {
    if (SM) return bpe_dyn[i];
    return __ldg(T.node + i);
}

// The state of one left-to-right pass: automaton node (and its record), the
// word length so far (capped at 63), and a ring of the last R token ids in
// shared memory (column `tid` of an R x NT array).
struct DpPass {
    uint4 nd;               // record of the current node
    unsigned state;
    int wd;
    unsigned short *ring;   // ring[i * NT]
};

// One step at symbol j (a base c): move the automaton, then take the first
// candidate (longest first) that starts the word or is compatible with the
// token before it.  The single base at the end of every list is taken
// without a check (no other candidate fits).  Returns (length << 16) | token.
template <int R, int NT, bool SM>
__device__ __forceinline__ unsigned dp_step(const BpeTables &T, DpPass &P, unsigned j, unsigned c) {
    P.state = node_next(P.nd, c);
    P.nd = node_at<SM>(T, P.state);
    if (P.wd < 63) ++P.wd;
    const int wd = P.wd;
    unsigned t1 = P.nd.z & 0xFFFFu, t2 = P.nd.z >> 16;
    int l1 = (int)(P.nd.w & 63u), l2 = (int)((P.nd.w >> 6) & 63u);
    // both candidates' checks are issued before either is used
    const bool n1 = (l1 != wd) && (l1 > 1);
    const bool n2 = (t2 != kNone16) && (l2 != wd) && (l2 > 1);
    const unsigned a1 = n1 ? P.ring[((j - l1) & (R - 1)) * NT] : 0u;
    const unsigned a2 = n2 ? P.ring[((j - l2) & (R - 1)) * NT] : 0u;
    const bool ok1 = !n1 || compat_bit(T.compat, T.V, a1, t1);
    const bool ok2 = !n2 || compat_bit(T.compat, T.V, a2, t2);
    if (ok1) return ((unsigned)l1 << 16) | t1;
    if (t2 != kNone16 && ok2) return ((unsigned)l2 << 16) | t2;
    // the rest of the list, two candidates per record
    unsigned nx = P.nd.w >> 16;
    unsigned last = ((unsigned)l2 << 16) | t2;
    for (int guard = 0; nx != kNone16 && guard < kMaxTokLen; ++guard) {
        const uint4 q = node_at<SM>(T, nx);
        t1 = q.z & 0xFFFFu;
        t2 = q.z >> 16;
        l1 = (int)(q.w & 63u);
        l2 = (int)((q.w >> 6) & 63u);
        if (l1 == wd || l1 == 1 ||
            compat_bit(T.compat, T.V, P.ring[((j - l1) & (R - 1)) * NT], t1))
            return ((unsigned)l1 << 16) | t1;
        last = ((unsigned)l1 << 16) | t1;
        if (t2 == kNone16) break;
        if (l2 == wd || l2 == 1 ||
            compat_bit(T.compat, T.V, P.ring[((j - l2) & (R - 1)) * NT], t2))
            return ((unsigned)l2 << 16) | t2;
        last = ((unsigned)l2 << 16) | t2;
        nx = q.w >> 16;
    }
    return last;  // unreachable for a valid table (the single base always fits)
}

template <bool SM>
__device__ __forceinline__ void dp_reset(const BpeTables &T, DpPass &P) {
    P.state = 0;
    P.nd = node_at<SM>(T, 0);
    P.wd = 0;
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

// One pass over symbols [j_begin, e) of segment `seg` (which starts at s),
// from the state in P (set up for j_begin).  Values before s go to the
// segment's halo, values from s on to W.tok; from s on the pass also carries
// F(j) = (exit << 24) | count: where the chain j -> j - |last(j)| first
// drops below s (offset s - 1 - exit position, < lmax) and how many tokens it
// holds until then.  At the end F of the last lmax positions is the
// segment's map.  `exact` turns true when the pass meets a true word start
// before s.  16 symbols per load and 16 values per pair of stores: s, H and
// the buffers are 16-aligned; j_begin only shifts where the first block
// starts.
template <int R, int NT, bool SM>
__device__ void seg_pass(const BpeTables &T, const BpeWork &W, long long seg, long long s,
                         long long e, long long j_begin, long long r, DpPass &P,
                         unsigned *ringf, bool &exact) {
    const long long nb = W.tot[1] + 1;
    long long next_b = (r + 1 < nb) ? W.rec_off[r + 1] : (1ll << 62);
    unsigned short *halo = W.halo + seg * (long long)W.H;
    const long long h0 = s - W.H;
    const unsigned N_ID = (unsigned)T.V;
    for (long long j0 = j_begin & ~15ll; j0 < e; j0 += 16) {
        const uint4 sv = *reinterpret_cast<const uint4 *>(W.sym + j0);
        // four values per 64-bit word; 0xFFFF: no value
        unsigned long long o0 = ~0ull, o1 = ~0ull, o2 = ~0ull, o3 = ~0ull;
        const int q0 = (j0 < j_begin) ? (int)(j_begin - j0) : 0;
        const int q1 = (e - j0 < 16) ? (int)(e - j0) : 16;
        // groups of four symbols: inside a group the shifts are constants
#pragma unroll 1
        for (int g = q0 >> 2; g < 4 && 4 * g < q1; ++g) {
            const unsigned wg = g == 0 ? sv.x : g == 1 ? sv.y : g == 2 ? sv.z : sv.w;
            unsigned long long grp = ~0ull;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int q = 4 * g + qq;
                if (q < q0 || q >= q1) continue;
                const long long j = j0 + q;
                while (j == next_b) {
                    dp_reset<SM>(T, P);
                    ++r;
                    next_b = (r + 1 < nb) ? W.rec_off[r + 1] : (1ll << 62);
                    if (j < s) exact = true;  // a record starts in the halo
                }
                const unsigned c = (wg >> (8 * qq)) & 0xFFu;
                const unsigned ju = (unsigned)j;  // ring slots: the low bits of j
                unsigned L, t;
                if (c >= 4) {
                    L = 1;
                    t = N_ID;
                    dp_reset<SM>(T, P);
                    if (j < s) exact = true;  // a word starts after it, before the segment
                } else {
                    const unsigned pk = dp_step<R, NT, SM>(T, P, ju, c);
                    L = pk >> 16;
                    t = pk & 0xFFFFu;
                }
                P.ring[(ju & (R - 1)) * NT] = (unsigned short)t;
                if (j >= s) {
                    const long long back = j - (long long)L;
                    const unsigned F = back < s ? ((unsigned)(s - 1 - back) << 24) | 1u
                                                : ringf[((unsigned)back & (R - 1)) * NT] + 1u;
                    ringf[(ju & (R - 1)) * NT] = F;
                }
                grp = (grp & ~(0xFFFFull << (16 * qq))) | ((unsigned long long)t << (16 * qq));
            }
            if (g == 0) o0 = grp;
            else if (g == 1) o1 = grp;
            else if (g == 2) o2 = grp;
            else o3 = grp;
        }
        const uint4 v0 = make_uint4((unsigned)o0, (unsigned)(o0 >> 32), (unsigned)o1,
                                    (unsigned)(o1 >> 32));
        const uint4 v1 = make_uint4((unsigned)o2, (unsigned)(o2 >> 32), (unsigned)o3,
                                    (unsigned)(o3 >> 32));
        uint4 *dst = (j0 >= s) ? reinterpret_cast<uint4 *>(W.tok + j0)
                               : reinterpret_cast<uint4 *>(halo + (j0 - h0));
        if (j0 >= s || W.H > 0) {
            dst[0] = v0;
            dst[1] = v1;
        }
    }
    if (j_begin < s) {
        // halo positions before the pass began hold no value
        for (long long x = h0; x < (j_begin & ~15ll); ++x) halo[x - h0] = (unsigned short)kNone16;
    }
    // the map: entry u (chain from e - 1 - u) -> (exit offset, tokens)
    unsigned first = 0xFFFFFFFFu;
    bool same = true;
    for (int u = 0; u < T.lmax; ++u) {
        const long long p = e - 1 - u;
        const unsigned F = (p >= s) ? ringf[(p & (R - 1)) * NT]
                                    : ((unsigned)(s - 1 - p) << 24);
        const unsigned v = F >> 24;
        W.map_v[seg * 32 + u] = (uint8_t)v;
        W.map_c[seg * 32 + u] = F & 0xFFFFFFu;
        if (u == 0) first = v;
        else if (v != first) same = false;
    }
    W.const_v[seg] = same ? (uint8_t)first : (uint8_t)0xFF;
}

// The merge pass, one segment per thread, started H symbols before it unless
// a word starts closer.  Persistent: NT threads per block, one block per SM,
// each thread takes segments tid, tid + grid threads, ...  Dynamic shared
// memory holds the automaton's node records (SM; 16 bytes each, loaded once
// per block) and the two rings of every thread.
template <int R, int NT, bool SM>
__global__ void __launch_bounds__(NT, 1) bpe_dp_kernel(BpeTables T, BpeWork W) {
    const int n_node_words = SM ? T.n_nodes : 0;
    unsigned short *ring_t = reinterpret_cast<unsigned short *>(bpe_dyn + n_node_words);
    unsigned *ring_f = reinterpret_cast<unsigned *>(ring_t + R * NT);
    if (SM) {
        for (int i = threadIdx.x; i < T.n_nodes; i += NT) bpe_dyn[i] = __ldg(T.node + i);
        __syncthreads();
    }
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0], n_rec = W.tot[1];
    if (n_rec + 1 > W.offsets_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_dev_status(W.status, DEV_CAPACITY);
        return;
    }
    const long long nb = n_rec + 1;
    for (long long seg = blockIdx.x * (long long)NT + threadIdx.x; seg * W.S < n_sym;
         seg += (long long)gridDim.x * NT) {
        const long long s = seg * W.S;
        const long long e = (s + W.S < n_sym) ? s + W.S : n_sym;
        long long r = rec_upper(W.rec_off, nb, s);
        long long a = s - W.H;
        bool exact = false;
        if (a <= W.rec_off[r]) {
            a = W.rec_off[r];
            exact = true;
        }
        while (r + 1 < nb && W.rec_off[r + 1] <= a) ++r;  // empty records at a
        DpPass P;
        P.ring = ring_t + threadIdx.x;
        dp_reset<SM>(T, P);
        seg_pass<R, NT, SM>(T, W, seg, s, e, a, r, P, ring_f + threadIdx.x, exact);
        W.flags[seg] = exact ? 1 : 0;
    }
}

template <int R, int NT, bool SM>
size_t dp_smem_bytes(int n_nodes) {
    return (SM ? (size_t)n_nodes * sizeof(uint4) : 0) + (size_t)R * NT * (2 + 4);
}

// A segment whose pass did not start exactly is correct if its halo agrees
// with its left neighbour's values over lmax consecutive symbols; the others
// are marked for repair.
__global__ void bpe_sync_kernel(BpeTables T, BpeWork W) {
    const long long seg = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (seg >= W.max_seg) return;
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0];
    const long long s = seg * W.S;
    uint8_t bad = 0;
    if (seg > 0 && s < n_sym && !W.flags[seg]) {
        const unsigned short *halo = W.halo + seg * (long long)W.H;
        int run = 0;
        bad = 1;
        for (long long j = s - W.H; j < s; ++j) {
            const unsigned short v = halo[j - (s - W.H)];
            run = (v != kNone16 && v == W.tok[j]) ? run + 1 : 0;
            if (run >= T.lmax) {
                bad = 0;
                break;
            }
        }
        if (bad) atomicAdd(W.n_bad, 1);
    }
    W.bad[seg] = bad;
}

// The segments to repair, in order, each with its region: the last exact
// segment at or before it.  Regions are independent (no chain of
// dependencies crosses an exact segment), so each region's segments are
// repaired by one thread, regions in parallel.  A pair scan over the
// segments (count of marked segments, last exact segment) gives both.
struct CntMax {
    long long c, m;
};
__device__ __forceinline__ CntMax cm_combine(CntMax a, CntMax b) {
    return CntMax{a.c + b.c, a.m > b.m ? a.m : b.m};
}
__device__ __forceinline__ CntMax cm_item(const BpeWork &W, long long i) {
    if (i >= W.max_seg) return CntMax{0, -1};
    return CntMax{W.bad[i], (i == 0 || W.flags[i]) ? i : -1};
}
// exclusive block scan of CntMax (identity {0, -1}); *total gets the block's reduction
__device__ __forceinline__ CntMax block_excl_scan_cm(CntMax v, CntMax *total) {
    __shared__ long long wc[kScanThreads / 32], wm[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    CntMax x = v;
    for (int o = 1; o < 32; o <<= 1) {
        CntMax y{__shfl_up_sync(0xffffffffu, x.c, o), __shfl_up_sync(0xffffffffu, x.m, o)};
        if (lane >= o) x = cm_combine(y, x);
    }
    if (lane == 31) {
        wc[warp] = x.c;
        wm[warp] = x.m;
    }
    __syncthreads();
    CntMax off{0, -1}, all{0, -1};
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const CntMax ww{wc[w], wm[w]};
        if (w < warp) off = cm_combine(off, ww);
        all = cm_combine(all, ww);
    }
    __syncthreads();
    *total = all;
    // exclusive within the warp: shift the inclusive value up by one lane
    CntMax ex{__shfl_up_sync(0xffffffffu, x.c, 1), __shfl_up_sync(0xffffffffu, x.m, 1)};
    if (lane == 0) ex = CntMax{0, -1};
    return cm_combine(off, ex);
}

__global__ void __launch_bounds__(kScanThreads) bpe_rep_reduce(BpeWork W) {
    if (*W.n_bad == 0) return;
    const long long i0 = (blockIdx.x * (long long)kScanThreads + threadIdx.x) * kScanItems;
    CntMax v{0, -1};
    for (int q = 0; q < kScanItems; ++q) v = cm_combine(v, cm_item(W, i0 + q));
    CntMax total;
    block_excl_scan_cm(v, &total);
    if (threadIdx.x == 0) {
        W.rep_sums[2 * blockIdx.x] = total.c;
        W.rep_sums[2 * blockIdx.x + 1] = total.m;
    }
}

__global__ void __launch_bounds__(kScanThreads) bpe_rep_top(BpeWork W, long long n_blocks) {
    if (*W.n_bad == 0) return;
    CntMax carry{0, -1};
    for (long long b0 = 0; b0 < n_blocks; b0 += kScanThreads) {
        const long long b = b0 + threadIdx.x;
        const CntMax v = (b < n_blocks) ? CntMax{W.rep_sums[2 * b], W.rep_sums[2 * b + 1]}
                                        : CntMax{0, -1};
        CntMax total;
        const CntMax ex = block_excl_scan_cm(v, &total);
        if (b < n_blocks) {
            const CntMax pre = cm_combine(carry, ex);
            W.rep_sums[2 * b] = pre.c;
            W.rep_sums[2 * b + 1] = pre.m;
        }
        carry = cm_combine(carry, total);
    }
}

__global__ void __launch_bounds__(kScanThreads) bpe_rep_down(BpeWork W) {
    if (*W.n_bad == 0) return;
    const long long i0 = (blockIdx.x * (long long)kScanThreads + threadIdx.x) * kScanItems;
    CntMax v{0, -1};
    for (int q = 0; q < kScanItems; ++q) v = cm_combine(v, cm_item(W, i0 + q));
    CntMax total;
    CntMax run = cm_combine(CntMax{W.rep_sums[2 * blockIdx.x], W.rep_sums[2 * blockIdx.x + 1]},
                            block_excl_scan_cm(v, &total));
    for (int q = 0; q < kScanItems; ++q) {
        const CntMax it = cm_item(W, i0 + q);
        run = cm_combine(run, CntMax{0, it.m});  // the region includes the item itself
        if (it.c) {
            W.rep_list[run.c] = (int)(i0 + q);
            W.rep_region[run.c] = (int)run.m;
        }
        run.c += it.c;
    }
}

// Exact recomputation of the marked segments.  One thread per region (the
// thread of the region's first listed segment) takes its segments in order:
// it rebuilds the pass state at the segment start from the (correct) values
// to its left, recomputes the segment (values and map), then re-checks the
// next segment against the new values and continues into it if it no longer
// agrees, up to the next exact segment.  Work per thread is bounded by its
// region; a region is one run of dependent segments.
template <int R>
__global__ void __launch_bounds__(kDpThreads) bpe_repair_kernel(BpeTables T, BpeWork W) {
    // global node records (repairs are rare); rings in static shared memory
    __shared__ unsigned short ring_t[R * kDpThreads];
    __shared__ unsigned ring_f[R * kDpThreads];
    const int nbad = *W.n_bad;
    const long long i = blockIdx.x * (long long)kDpThreads + threadIdx.x;
    if (nbad == 0 || i >= nbad) return;
    if (dev_failed(W.status)) return;
    const int region = W.rep_region[i];
    if (i > 0 && W.rep_region[i - 1] == region) return;  // not the region's first
    const long long n_sym = W.tot[0], nb = W.tot[1] + 1;
    DpPass P;
    P.ring = ring_t + threadIdx.x;
    unsigned *ringf = ring_f + threadIdx.x;
    long long done_until = 0;  // symbols below this are final
    for (long long k = i; k < nbad && W.rep_region[k] == region; ++k) {
        long long seg = W.rep_list[k];
        long long s = seg * W.S;
        if (s < done_until) continue;
        while (true) {
            // pass state at s from the values to its left
            long long r = rec_upper(W.rec_off, nb, s);
            while (r + 1 < nb && W.rec_off[r + 1] <= s) ++r;
            const long long ws = W.rec_off[r];
            long long x = s - 1;
            while (x >= ws && x >= s - 63 && W.sym[x] < 4) --x;
            // symbols (x, s) are the word so far (capped at 63)
            dp_reset<false>(T, P);
            const long long from = (s - (x + 1) > T.lmax) ? s - T.lmax : x + 1;
            for (long long y = from; y < s; ++y) {
                P.state = node_next(P.nd, W.sym[y]);
                P.nd = node_at<false>(T, P.state);
            }
            P.wd = (int)(s - (x + 1));
            for (long long y = (s - R > 0 ? s - R : 0); y < s; ++y)
                P.ring[(y & (R - 1)) * kDpThreads] = W.tok[y];
            const long long e = (s + W.S < n_sym) ? s + W.S : n_sym;
            bool exact = true;
            seg_pass<R, kDpThreads, false>(T, W, seg, s, e, s, r, P, ringf, exact);
            done_until = e;
            ++seg;
            s = seg * W.S;
            if (s >= n_sym || W.flags[seg]) break;
            // does the next segment's fresh pass agree with the new values?
            const unsigned short *halo = W.halo + seg * (long long)W.H;
            int run = 0;
            bool ok = false;
            for (long long j = s - W.H; j < s && !ok; ++j) {
                const unsigned short v = halo[j - (s - W.H)];
                run = (v != kNone16 && v == W.tok[j]) ? run + 1 : 0;
                ok = run >= T.lmax;
            }
            if (ok) break;
        }
    }
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

// The ids of every segment, in two phases per block of kEmitT segments:
// (1) each thread walks its segment's chain from the true entry backwards and
// marks the token ends in a shared-memory bitmap (tok values read in windows
// of 32 positions, four independent 16-byte loads held in registers, so one
// global round trip serves about six tokens); (2) each warp then writes its
// 32 segments one after another: lane w takes bitmap word w (32 positions),
// a warp scan of the counts gives each lane its output run, and the warp's
// loads of tok and stores of ids are coalesced.  Segments longer than
// kEmitMaxS use emit_walk_kernel, which writes each id as it walks.
constexpr int kEmitT = 128;
constexpr int kEmitMaxS = 1024;  // the default segment; longer ones take bpe_emit_walk_kernel

__device__ __forceinline__ unsigned pick4(const uint4 &v, int i) {
    return i < 2 ? (i == 0 ? v.x : v.y) : (i == 2 ? v.z : v.w);
}

// Walk a segment's chain: f(e, t) for every token (end e, id t), last first.
// Tokens are at most 32 symbols long, so the walk goes through the 32-position
// windows of tok strictly one after another, downwards: the window below the
// current one is loaded one window ahead, and its round trip overlaps the
// tokens of the current one.
template <class F>
__device__ __forceinline__ void walk_chain(const BpeTables &T, const BpeWork &W, long long s,
                                           long long e, F &&f) {
    if (e < s) return;
    const long long floor_w = s & ~31ll;  // the lowest window the walk can reach
    long long wb = e & ~31ll;             // first position of the window held
    const uint4 *src = reinterpret_cast<const uint4 *>(W.tok + wb);
    uint4 v0 = src[0], v1 = src[1], v2 = src[2], v3 = src[3];
    uint4 p0 = make_uint4(0, 0, 0, 0), p1 = p0, p2 = p0, p3 = p0;
    if (wb - 32 >= floor_w) {
        const uint4 *q = src - 4;
        p0 = q[0];
        p1 = q[1];
        p2 = q[2];
        p3 = q[3];
    }
    while (e >= s) {
        if (e < wb) {  // the next window down, already loaded; load the one below it
            wb -= 32;
            v0 = p0;
            v1 = p1;
            v2 = p2;
            v3 = p3;
            if (wb - 32 >= floor_w) {
                const uint4 *q = reinterpret_cast<const uint4 *>(W.tok + wb - 32);
                p0 = q[0];
                p1 = q[1];
                p2 = q[2];
                p3 = q[3];
            }
        }
        const int wi = (int)((e - wb) >> 1);  // 32-bit word of the window, 0..15
        const unsigned w = wi < 8 ? (wi < 4 ? pick4(v0, wi) : pick4(v1, wi - 4))
                                  : (wi < 12 ? pick4(v2, wi - 8) : pick4(v3, wi - 12));
        const unsigned t = (e & 1) ? (w >> 16) : (w & 0xFFFFu);
        f(e, t);
        e -= __ldg(T.tok_len + t);
    }
}

__global__ void __launch_bounds__(kEmitT) bpe_emit_kernel(BpeTables T, BpeWork W) {
    __shared__ unsigned bm[kEmitMaxS / 32][kEmitT + 1];  // [word][segment of the block], padded
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0];
    const long long n_seg = (n_sym + W.S - 1) / W.S;
    const int words = (W.S + 31) / 32;
    const long long seg0 = blockIdx.x * (long long)kEmitT;
    // 1. token ends of this thread's segment
    {
        const long long seg = seg0 + tid;
        for (int w = 0; w < words; ++w) bm[w][tid] = 0u;
        if (seg < n_seg) {
            const long long s = seg * W.S;
            const long long e_end = (s + W.S < n_sym) ? s + W.S : n_sym;
            walk_chain(T, W, s, e_end - 1 - W.entry[seg], [&](long long e, unsigned) {
                const int x = (int)(e - s);
                bm[x >> 5][tid] |= 1u << (x & 31);
            });
        }
    }
    __syncthreads();
    // 2. each warp writes its 32 segments' ids, one segment at a time
    for (int i = 0; i < 32; ++i) {
        const int col = warp * 32 + i;
        const long long seg = seg0 + col;
        if (seg >= n_seg) break;
        const long long s = seg * W.S;
        long long out = W.base[seg];
        for (int w0 = 0; w0 < words; w0 += 32) {
            const int w = w0 + lane;
            const unsigned bits = (w < words) ? bm[w][col] : 0u;
            const unsigned c = __popc(bits);
            unsigned x = c;  // inclusive scan of the counts over the warp
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            long long pos = out + (x - c);
            unsigned m = bits;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const unsigned id = W.tok[s + 32ll * w + b];
                if (pos >= 0 && pos < W.out_cap) W.out[pos] = (int)id;
                ++pos;
            }
            out += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

// Long segments: thread per segment, each id written as the chain is walked.
__global__ void __launch_bounds__(256) bpe_emit_walk_kernel(BpeTables T, BpeWork W) {
    const long long seg = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (dev_failed(W.status)) return;
    const long long n_sym = W.tot[0];
    const long long n_seg = (n_sym + W.S - 1) / W.S;
    if (seg >= n_seg) return;
    const long long s = seg * W.S;
    const long long e_end = (s + W.S < n_sym) ? s + W.S : n_sym;
    long long pos = W.base[seg] + W.count[seg];
    walk_chain(T, W, s, e_end - 1 - W.entry[seg], [&](long long, unsigned t) {
        --pos;
        if (pos >= 0 && pos < W.out_cap) W.out[pos] = (int)t;
    });
}

// Record starts (in symbols) -> record starts (in ids), in place.
__global__ void bpe_offsets_kernel(BpeTables T, BpeWork W) {
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
                e -= __ldg(T.tok_len + W.tok[e]);
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
    int M = 0, V = 0, lmax = 1, n_nodes = 1;
    uint4 *d_node = nullptr;
    uint8_t *d_tok_len = nullptr;
    unsigned *d_compat = nullptr;
    int S = 1024, H = 64;

    // workspace
    long long cap_bytes = -1;
    uint8_t *d_sym = nullptr, *d_flags = nullptr, *d_bad = nullptr;
    unsigned short *d_tok = nullptr, *d_halo = nullptr;
    uint8_t *d_map_v = nullptr, *d_const = nullptr, *d_entry = nullptr;
    unsigned *d_map_c = nullptr;
    unsigned *d_count = nullptr;
    long long *d_base = nullptr, *d_bsums = nullptr, *d_rsums = nullptr, *d_tot = nullptr;
    int *d_nbad = nullptr, *d_rep_list = nullptr, *d_rep_region = nullptr;
    long long seg_cap = 0;
    int ws_S = 0, ws_H = 0;
};

namespace {

void free_workspace(BpeState *b) {
    void *p[] = {b->d_sym, b->d_flags, b->d_bad, b->d_tok, b->d_halo, b->d_map_v, b->d_const,
                 b->d_entry, b->d_map_c, b->d_count, b->d_base, b->d_bsums, b->d_rsums, b->d_tot,
                 b->d_nbad, b->d_rep_list, b->d_rep_region};
    for (void *q : p) cudaFree(q);
    b->d_sym = b->d_flags = b->d_bad = nullptr;
    b->d_tok = b->d_halo = nullptr;
    b->d_map_v = b->d_const = b->d_entry = nullptr;
    b->d_map_c = b->d_count = nullptr;
    b->d_base = b->d_bsums = b->d_rsums = b->d_tot = nullptr;
    b->d_nbad = b->d_rep_list = b->d_rep_region = nullptr;
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
    size_t sz[] = {(size_t)cap + 16,                  // sym
                   (size_t)nseg,                      // flags
                   (size_t)nseg,                      // bad
                   2 * ((size_t)cap + 16),            // tok
                   2 * ((size_t)nseg * b->H + 16),    // halo
                   (size_t)nseg * 32,                 // map_v
                   (size_t)nseg,                      // const
                   (size_t)nseg,                      // entry
                   (size_t)nseg * 32 * 4,             // map_c
                   (size_t)nseg * 4,                  // count
                   (size_t)(nseg + 1) * 8,            // base
                   (size_t)nblk * 8,                  // block sums
                   (size_t)nblk * 16,                 // repair listing block sums
                   16,                                // tot
                   16,                                // n_bad
                   (size_t)nseg * 4,                  // repair list
                   (size_t)nseg * 4};                 // repair regions
    void **ptr[] = {(void **)&b->d_sym,     (void **)&b->d_flags,   (void **)&b->d_bad,
                    (void **)&b->d_tok,     (void **)&b->d_halo,    (void **)&b->d_map_v,
                    (void **)&b->d_const,   (void **)&b->d_entry,   (void **)&b->d_map_c,
                    (void **)&b->d_count,   (void **)&b->d_base,    (void **)&b->d_bsums,
                    (void **)&b->d_rsums,   (void **)&b->d_tot,     (void **)&b->d_nbad,
                    (void **)&b->d_rep_list, (void **)&b->d_rep_region};
    for (int i = 0; i < 17; ++i) {
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
    // Aho-Corasick automaton over the strings of the self-encoding tokens:
    // trie (node 0 = root), failure links by breadth-first order, complete
    // transitions, and for every node the list of its candidates -- the
    // self-encoding tokens that are suffixes of its string, longest first.
    std::vector<unsigned> ch(4, 0);
    std::vector<int> term(1, -1), depth(1, 0);
    int lmax = 1;
    for (int t = 0; t < V; ++t) {
        if (!self[t]) continue;
        lmax = std::max(lmax, len[t]);
        unsigned node = 0;
        for (int d = 0; d < len[t]; ++d) {
            const unsigned c = str[t][d];
            if (!ch[node * 4 + c]) {
                ch[node * 4 + c] = (unsigned)term.size();
                term.push_back(-1);
                depth.push_back(depth[node] + 1);
                ch.insert(ch.end(), {0, 0, 0, 0});
            }
            node = ch[node * 4 + c];
        }
        term[node] = t;
    }
    const size_t N = term.size();
    if (N >= 0xFFFF) {
        cleanup();
        return fail(h, DNATOK_ERR_TABLE, "BPE token automaton exceeds 65534 nodes");
    }
    std::vector<unsigned> fail_(N, 0), delta(N * 4, 0), order;
    order.reserve(N);
    order.push_back(0);
    for (size_t qi = 0; qi < order.size(); ++qi) {
        const unsigned u = order[qi];
        for (unsigned c = 0; c < 4; ++c) {
            const unsigned v = ch[u * 4 + c];
            if (v) {
                fail_[v] = (u == 0) ? 0 : delta[fail_[u] * 4 + c];
                delta[u * 4 + c] = v;
                order.push_back(v);
            } else {
                delta[u * 4 + c] = (u == 0) ? 0 : delta[fail_[u] * 4 + c];
            }
        }
    }
    // dict[u]: the nearest proper suffix node that is a token (or none)
    std::vector<unsigned> dict(N, kNone16);
    for (size_t qi = 1; qi < order.size(); ++qi) {
        const unsigned u = order[qi], f = fail_[u];
        dict[u] = (f != 0 && term[f] >= 0) ? f : dict[f];
    }
    std::vector<uint4> rec(N);
    for (size_t u = 0; u < N; ++u) {
        const unsigned c1 = (term[u] >= 0) ? (unsigned)u : dict[u];
        const unsigned c2 = (c1 != kNone16) ? dict[c1] : kNone16;
        const unsigned c3 = (c2 != kNone16) ? dict[c2] : kNone16;
        const unsigned t1 = c1 != kNone16 ? (unsigned)term[c1] : kNone16;
        const unsigned t2 = c2 != kNone16 ? (unsigned)term[c2] : kNone16;
        const unsigned l1 = c1 != kNone16 ? (unsigned)depth[c1] : 0u;
        const unsigned l2 = c2 != kNone16 ? (unsigned)depth[c2] : 0u;
        rec[u].x = delta[u * 4 + 0] | (delta[u * 4 + 1] << 16);
        rec[u].y = delta[u * 4 + 2] | (delta[u * 4 + 3] << 16);
        rec[u].z = t1 | (t2 << 16);
        rec[u].w = l1 | (l2 << 6) | (c3 << 16);
    }
    std::vector<uint8_t> tl(V + 1);
    for (int t = 0; t < V; ++t) tl[t] = (uint8_t)std::min(len[t], 255);
    tl[V] = 1;  // N_ID
    b->lmax = lmax;
    b->n_nodes = (int)N;
    b->H = std::max(64, ((4 * lmax + 15) / 16) * 16);
    const unsigned long long nbits = (unsigned long long)V * V;
    const size_t cwords = (size_t)((nbits + 31) / 32) + 2;
    e = cudaMalloc(&b->d_node, sizeof(uint4) * N);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tok_len, V + 1);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_compat, cwords * 4);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_node, rec.data(), sizeof(uint4) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tok_len, tl.data(), V + 1, cudaMemcpyHostToDevice);
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
    cudaFree(b->d_node);
    cudaFree(b->d_tok_len);
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

dnatok_status bpe_get_launch(const dnatok_handle *h, int *seg_symbols, int *halo) {
    if (!h->bpe) return DNATOK_ERR_STATE;
    *seg_symbols = h->bpe->S;
    *halo = h->bpe->H;
    return DNATOK_OK;
}

dnatok_status bpe_stats(dnatok_handle *h, long long *out, cudaStream_t s) {
    BpeState *b = h->bpe;
    if (!b) return fail(h, DNATOK_ERR_STATE, "not a BPE handle");
    out[0] = out[1] = out[2] = 0;
    if (!b->d_tot || !b->d_nbad) return DNATOK_OK;  // nothing encoded yet
    long long tot[2] = {0, 0};
    int bad = 0;
    cudaError_t e = cudaMemcpyAsync(tot, b->d_tot, sizeof(tot), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, b->d_nbad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e, "BPE statistics read");
    out[0] = tot[0];
    out[1] = (tot[0] + b->ws_S - 1) / (b->ws_S > 0 ? b->ws_S : 1);
    out[2] = bad;
    return DNATOK_OK;
}

// The merge pass launch: ring depth by the longest token, the node table in
// shared memory when it fits beside the rings, one persistent block per SM.
template <int R, int NT, bool SM>
static cudaError_t launch_dp_as(const BpeTables &T, const BpeWork &W, int sm_count,
                                cudaStream_t s) {
    const size_t smem = dp_smem_bytes<R, NT, SM>(T.n_nodes);
    static size_t attr = 0;
    if (attr < smem) {
        const cudaError_t e = cudaFuncSetAttribute(bpe_dp_kernel<R, NT, SM>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    long long grid = (W.max_seg + NT - 1) / NT;
    if (grid > sm_count) grid = sm_count;
    if (grid < 1) grid = 1;
    bpe_dp_kernel<R, NT, SM><<<(unsigned)grid, NT, smem, s>>>(T, W);
    return cudaGetLastError();
}

static cudaError_t launch_dp(dnatok_handle *h, const BpeTables &T, const BpeWork &W,
                             cudaStream_t s) {
    constexpr size_t kSmemMax = 220 * 1024;
    if (T.lmax <= 16) {
        if (dp_smem_bytes<16, 1024, true>(T.n_nodes) <= kSmemMax)
            return launch_dp_as<16, 1024, true>(T, W, h->sm_count, s);
        return launch_dp_as<16, 1024, false>(T, W, h->sm_count, s);
    }
    if (dp_smem_bytes<32, 512, true>(T.n_nodes) <= kSmemMax)
        return launch_dp_as<32, 512, true>(T, W, h->sm_count, s);
    return launch_dp_as<32, 512, false>(T, W, h->sm_count, s);
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
    cudaError_t e = cudaMemsetAsync(b->d_nbad, 0, sizeof(int), s);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemsetAsync");

    BpeTables T{b->V, b->lmax, b->n_nodes, b->d_node, b->d_tok_len, b->d_compat};
    BpeWork W;
    std::memset(&W, 0, sizeof(W));
    W.sym = b->d_sym;
    W.tok = b->d_tok;
    W.halo = b->d_halo;
    W.flags = b->d_flags;
    W.bad = b->d_bad;
    W.map_v = b->d_map_v;
    W.map_c = b->d_map_c;
    W.const_v = b->d_const;
    W.count = b->d_count;
    W.entry = b->d_entry;
    W.base = b->d_base;
    W.block_sums = b->d_bsums;
    W.rep_sums = b->d_rsums;
    W.n_bad = b->d_nbad;
    W.rep_list = b->d_rep_list;
    W.rep_region = b->d_rep_region;
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

    const unsigned gdp = (unsigned)((W.max_seg + kDpThreads - 1) / kDpThreads);
    const unsigned g128 = (unsigned)((W.max_seg + 127) / 128);
    const unsigned g256 = (unsigned)((W.max_seg + 255) / 256);
    const long long nblk = scan_blocks(W.max_seg);
    e = launch_dp(h, T, W, s);
    if (e != cudaSuccess) return fail_cuda(h, e, "BPE merge pass launch");
    bpe_sync_kernel<<<g128, 128, 0, s>>>(T, W);
    bpe_rep_reduce<<<(unsigned)nblk, kScanThreads, 0, s>>>(W);
    bpe_rep_top<<<1, kScanThreads, 0, s>>>(W, nblk);
    bpe_rep_down<<<(unsigned)nblk, kScanThreads, 0, s>>>(W);
    if (b->lmax <= 16) bpe_repair_kernel<16><<<gdp, kDpThreads, 0, s>>>(T, W);
    else bpe_repair_kernel<32><<<gdp, kDpThreads, 0, s>>>(T, W);
    bpe_entries_kernel<<<g128, 128, 0, s>>>(T, W);
    bpe_scan_reduce<<<(unsigned)nblk, kScanThreads, 0, s>>>(W);
    bpe_scan_top<<<1, kScanThreads, 0, s>>>(W, nblk);
    bpe_scan_down<<<(unsigned)nblk, kScanThreads, 0, s>>>(W);
    // the emit takes its positions from the scans: launch it only if they launched
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e, "BPE kernel launch");
    if (b->S <= kEmitMaxS)
        bpe_emit_kernel<<<(unsigned)((W.max_seg + kEmitT - 1) / kEmitT), kEmitT, 0, s>>>(T, W);
    else
        bpe_emit_walk_kernel<<<g256, 256, 0, s>>>(T, W);
    const long long nrec_bound = raw ? n_seq + 1 : offsets_capacity;
    long long og = (nrec_bound + 255) / 256;
    if (og > 4096) og = 4096;
    if (og < 1) og = 1;
    bpe_offsets_kernel<<<(unsigned)og, 256, 0, s>>>(T, W);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e, "BPE kernel launch");
    return DNATOK_OK;
}

}  // namespace dnatok
