// ktab_direct.cu -- table-driven k-mers straight from RAW bytes without
// separators.
//
// When no byte of the input is below 0x21, every byte is a kept symbol:
// symbol j of the input is byte j, a record of L bytes has ceil(L / k)
// windows (Algorithm 2 cuts it into windows of k from its start), and the
// window plan (direct_plan_kernel with a tile map) gives, before any byte is
// read, the window offsets of the records and, for every tile of kKW
// windows, the record holding its first window.
// Only a window's token count needs the data -- 1 for a table entry, k for a
// whole window without one, L mod k for a tail -- so the encode is
//   1. the window plan (one block);
//   2. kd_count_kernel: each CTA a contiguous run of tiles; every window's
//      table entry (or a mark: how many single-symbol ids it expands to) to
//      a window array, the tile's token count to tsum[tile];
//   3. tile_scan_kernel (one block): tile offsets, totals, the offsets of
//      records with no window left;
//   4. kd_expand_kernel: the window entries to ids at the tile offsets (the
//      few windows without an entry read their bytes again), and the record
//      offsets.
// No tile waits on another.  Within a count CTA the next tile's bytes are
// on their way by TMA bulk copy (into the second of two shared buffers)
// while the current tile is counted; once they land they are turned into
// digits (A0 C1 G2 T3, 4 for every other byte) in place.  A byte below 0x21
// raises the gate: the general path behind these kernels (symbol pass,
// window offsets, count, scan, emit) then redoes the encode.  Traffic: the
// input once, the window entries twice (2 B each for k <= 6 with every id
// below 0x8000, else 4 B) and the ids once, against a symbol plane written
// once and read twice by the general path.
#include <atomic>
#include <cstring>

#include "handle.h"
#include "ktab.cuh"

namespace dnatok {
namespace {

struct KdParams {
    const uint8_t *base;          // input bytes rounded down to 16
    int head_pad;                 // input - base
    long long n;                  // input bytes
    const long long *so;          // seq_offsets (n_seq + 1)
    long long n_seq;
    const long long *wpre;        // window offsets from the plan (n_seq + 1)
    const long long *tile_rec;    // per tile: record of its first window
    long long *tsum;              // per tile: token count (count), offset (expand)
    void *went;                   // per window: entry (u16 or int32, see KdEnt)
    const int *klut;              // kmer_lut (5^k)
    const uint16_t *klut16;       // the same as u16 (0xFFFF: no entry), or null
    KtabIds ids;                  // base_ids
    int *out;
    long long ids_cap;
    long long *id_offsets;
    unsigned *gate;
    unsigned epoch;
    int *status;
};

// Digit of each byte of a word: A0 C1 G2 T3 (either case), 4 for any other
// byte.  A byte is one of ACGTacgt iff its bits 0, 3, 4, 6 and 7 match those
// of 'A', or those of 'T' (bit 2 set, bit 1 clear) for a T; the code is
// bit1 ^ bit2 in bit 0 and bit2 ^ bit3 in bit 1.
__device__ __forceinline__ unsigned kd_digits4(unsigned x) {
    const unsigned s1 = x >> 1, s2 = x >> 2;
    const unsigned code = (s1 ^ s2) & 0x03030303u;
    const unsigned t = s2 & ~s1 & 0x01010101u;
    const unsigned v = (x & 0xD9D9D9D9u) ^ (t * 0x0Fu + 0x41414141u);  // zero byte: a base
    const unsigned nz = (((v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | v) & 0x80808080u;
    const unsigned nm = (nz >> 7) * 0xFFu;
    return (code & ~nm) | (0x04040404u & nm);
}

// 0x80 in every byte of the word below 0x21
__device__ __forceinline__ unsigned kd_low4(unsigned x) {
    return ~((x | 0x80808080u) - 0x21212121u) & ~x & 0x80808080u;
}

// Turn the raw bytes of a landed tile into digits in place: s holds the
// 16-byte aligned span around bytes [lead, lead + n).  Sets `low` when a
// byte of that range is below 0x21.
__device__ __forceinline__ void kd_digitize(uint8_t *s, int lead, int n, int tid, bool &low) {
    uint4 *v = reinterpret_cast<uint4 *>(s);
    const int end = lead + n;
    const int chunks = (end + 15) >> 4;
    for (int c = tid; c < chunks; c += kKThreads) {
        const uint4 w = v[c];
        if (kd_low4(w.x) | kd_low4(w.y) | kd_low4(w.z) | kd_low4(w.w)) {
            // rare: a byte below 0x21 in the chunk, perhaps outside the range
            const unsigned b[4] = {w.x, w.y, w.z, w.w};
            for (int j = 0; j < 16; ++j) {
                const int x = 16 * c + j;
                if (x >= lead && x < end && ((b[j >> 2] >> (8 * (j & 3))) & 0xFFu) < 0x21u)
                    low = true;
            }
        }
        v[c] = make_uint4(kd_digits4(w.x), kd_digits4(w.y), kd_digits4(w.z), kd_digits4(w.w));
    }
}

// Where a tile's bytes are: its first window's record and its byte range
// [jlo, jhi).
struct KdMeta {
    long long rb, jlo, jhi;
};

// The first byte of window w of record r.
__device__ __forceinline__ long long kd_window_byte(const KdParams &p, long long r, long long w,
                                                   int k) {
    return p.so[r] + (w - p.wpre[r]) * k;
}

__device__ __forceinline__ KdMeta kd_meta(const KdParams &p, long long t, long long n_tiles,
                                          int k) {
    KdMeta m;
    m.rb = p.tile_rec[t];
    const long long r1 = (t + 1 < n_tiles) ? p.tile_rec[t + 1] : 0;
    m.jlo = kd_window_byte(p, m.rb, t * kKW, k);
    m.jhi = (t + 1 < n_tiles) ? kd_window_byte(p, r1, (t + 1) * kKW, k) : p.n;
    return m;
}

// Start the bulk copy of tile m's bytes into the shared buffer s (thread 0):
// the 16-byte aligned span [a0 & ~15, a1 rounded up to 16) of the input,
// a0 = head_pad + jlo, a1 = head_pad + jhi, which ends inside the input's
// last 16-byte granule (at most cap bytes).  The caller's barrier and the
// proxy fence order it after every earlier read of s by this CTA.
__device__ __forceinline__ void kd_issue(const KdParams &p, const KdMeta &m, uint8_t *s,
                                         uint64_t *bar, long long cap) {
    const long long a0 = (long long)p.head_pad + m.jlo, a1 = (long long)p.head_pad + m.jhi;
    const long long lo = a0 & ~15ll;
    long long bytes = ((a1 + 15) & ~15ll) - lo;
    if (bytes > cap) bytes = cap;  // (malformed input)
    fence_proxy_async_shared();
    if (bytes > 0) {
        mbar_arrive_expect_tx(bar, (unsigned)bytes);
        tma_load_1d(s, p.base + lo, (unsigned)bytes, bar);
    } else {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
    }
}

// A bounded wait for a bulk copy: false when it has not landed after
// kSpinLimit polls.  Each poll lets the thread sleep up to 20 us while the
// copy is in flight, so waiting warps take no issue slots from the others.
__device__ __forceinline__ bool kd_wait(uint64_t *bar, unsigned parity) {
    int spins = 0;
    while (!mbar_try_wait_hint(bar, parity, 20000u))
        if (++spins > kSpinLimit) return false;
    return true;
}

__device__ __forceinline__ int kd_nsym(const KdMeta &m, int K) {
    long long n = m.jhi - m.jlo;
    if (n > (long long)kKW * K) n = (long long)kKW * K;  // (malformed input)
    return n < 0 ? 0 : (int)n;
}


// A window's entry for the expand pass: its id; for a whole window without
// a table entry, its base-5 index (its K digits); for a record's tail of c
// symbols, c and their base-5 index.  Tails of fewer symbols come first:
// kd_off(c) = (5^c - 1) / 4 indices before the tails of c symbols.
//   u16 (K <= 6, every id below 0x8000): id; 0xC000 + index;
//       0x8000 + kd_off(c) + index
//   int32: id; -1 - index; -1 - 5^K - (kd_off(c) + index)
__host__ __device__ constexpr int kd_off(int c) { return (pow5(c) - 1) / 4; }

template <typename E, int K>
struct KdEnt;
template <int K>
struct KdEnt<uint16_t, K> {
    static __device__ __forceinline__ uint16_t id(int v) { return (uint16_t)v; }
    static __device__ __forceinline__ uint16_t whole(int index) { return (uint16_t)(0xC000 + index); }
    static __device__ __forceinline__ uint16_t tail(int c, int index) {
        return (uint16_t)(0x8000 + kd_off(c) + index);
    }
    static __device__ __forceinline__ bool is_id(uint16_t e) { return e < 0x8000u; }
    // ids the entry stands for (the tail's length found only for a tail)
    static __device__ __forceinline__ int count(uint16_t e) {
        if (e < 0x8000u) return 1;
        if (e >= 0xC000u) return K;
        int v;
        return tail_decode((int)e - 0x8000, v);
    }
    // ids the entry stands for; v = the id (is_id) or the digits' index
    static __device__ __forceinline__ int decode(uint16_t e, int &v, bool &is_id) {
        is_id = e < 0x8000u;
        if (is_id) {
            v = e;
            return 1;
        }
        if (e >= 0xC000u) {
            v = e - 0xC000;
            return K;
        }
        return tail_decode((int)e - 0x8000, v);
    }
    static __device__ __forceinline__ int tail_decode(int u, int &v) {
        int c = 0;
#pragma unroll
        for (int x = 1; x < K; ++x)
            if (kd_off(x) <= u) c = x;
        v = u - kd_off(c);
        return c;
    }
};
template <int K>
struct KdEnt<int, K> {
    static __device__ __forceinline__ int id(int v) { return v; }
    static __device__ __forceinline__ int whole(int index) { return -1 - index; }
    static __device__ __forceinline__ int tail(int c, int index) {
        return -1 - pow5(K) - (kd_off(c) + index);
    }
    static __device__ __forceinline__ bool is_id(int e) { return e >= 0; }
    static __device__ __forceinline__ int count(int e) {
        if (e >= 0) return 1;
        const int u = -1 - e;
        if (u < pow5(K)) return K;
        int v;
        return KdEnt<uint16_t, K>::tail_decode(u - pow5(K), v);
    }
    static __device__ __forceinline__ int decode(int e, int &v, bool &is_id) {
        is_id = e >= 0;
        if (is_id) {
            v = e;
            return 1;
        }
        const int u = -1 - e;
        if (u < pow5(K)) {
            v = u;
            return K;
        }
        return KdEnt<uint16_t, K>::tail_decode(u - pow5(K), v);
    }
};

// Store a thread's kKPer entries (consecutive windows from a multiple of
// kKPer, so the store is 16-byte aligned).
__device__ __forceinline__ void kd_store_ents(uint16_t *dst, const uint16_t (&e)[kKPer]) {
    *reinterpret_cast<uint4 *>(dst) =
        make_uint4(e[0] | ((unsigned)e[1] << 16), e[2] | ((unsigned)e[3] << 16),
                   e[4] | ((unsigned)e[5] << 16), e[6] | ((unsigned)e[7] << 16));
}
__device__ __forceinline__ void kd_store_ents(int *dst, const int (&e)[kKPer]) {
    reinterpret_cast<int4 *>(dst)[0] = make_int4(e[0], e[1], e[2], e[3]);
    reinterpret_cast<int4 *>(dst)[1] = make_int4(e[4], e[5], e[6], e[7]);
}
__device__ __forceinline__ void kd_load_ents(const uint16_t *src, uint16_t (&e)[kKPer]) {
    const uint4 v = *reinterpret_cast<const uint4 *>(src);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < kKPer; ++q) e[q] = (uint16_t)(w[q >> 1] >> (16 * (q & 1)));
}
__device__ __forceinline__ void kd_load_ents(const int *src, int (&e)[kKPer]) {
    const int4 a = reinterpret_cast<const int4 *>(src)[0];
    const int4 b = reinterpret_cast<const int4 *>(src)[1];
    e[0] = a.x; e[1] = a.y; e[2] = a.z; e[3] = a.w;
    e[4] = b.x; e[5] = b.y; e[6] = b.z; e[7] = b.w;
}

// The entry of a window from the per-window walk (t_sym: the tile's digits).
template <typename E, int K>
__device__ __forceinline__ E kd_entry(const KWin &a, const uint8_t *t_sym) {
    if (a.ent >= 0 && a.cnt == 1) return KdEnt<E, K>::id(a.ent);
    if (a.cnt == K) return KdEnt<E, K>::whole(a.idx);
    int index = 0;  // a tail (or nothing): its digits' index
    for (int y = 0; y < a.cnt; ++y) index = index * 5 + t_sym[a.j + y];
    return KdEnt<E, K>::tail(a.cnt, index);
}

// The count pass: a contiguous run of tiles of windows per CTA; per tile its
// token count to tsum[tile] and every window's entry to went.  Each thread
// takes kKPer consecutive windows of the tile, as the two-pass kernels over
// the symbol plane do; the tile's bytes and record window sit in one of two
// shared buffers while the next tile's bytes arrive in the other; once they
// land they become digits in place.  T16: the table in shared memory as
// u16.
template <int K, bool T16, typename E>
__global__ void __launch_bounds__(kKThreads, 3) kd_count_kernel(const KdParams p) {
    constexpr long long kSym = ktab_sym_bytes(K);
    extern __shared__ __align__(16) uint8_t dyn[];
    uint16_t *s_tab = reinterpret_cast<uint16_t *>(dyn);
    uint8_t *s_buf = dyn + ktab_tab_bytes(K, T16);  // two tiles of kSym bytes
    __shared__ long long s_wp[2][kKRW + 1], s_sr[2][kKRW + 1];
    __shared__ KdMeta s_meta[2];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int s_wsum[kKThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    E *went = static_cast<E *>(p.went);
    if (T16) {  // the table was written when the handle was made: load it before the plan ends
        const uint4 *src = reinterpret_cast<const uint4 *>(p.klut16);
        uint4 *dst = reinterpret_cast<uint4 *>(s_tab);
        for (int c = tid; c < ktab_tab_bytes(K, T16) / 16; c += kKThreads) dst[c] = src[c];
    }
    pdl_wait();  // the plan has finished and its writes are visible
    if (*(volatile const unsigned *)p.gate == p.epoch) return;  // it declined the offsets
    const long long n_rec = p.n_seq;
    const long long n_win = p.wpre[n_rec];
    const long long n_tiles = (n_win + kKW - 1) / kKW;
    const long long t_begin = (long long)blockIdx.x * n_tiles / gridDim.x;
    const long long t_end = (long long)(blockIdx.x + 1) * n_tiles / gridDim.x;
    if (t_begin >= t_end) return;
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phase[2] = {0u, 0u};
    bool low = false, failed = false;
    KdMeta nx{0, 0, 0};  // thread 0: the tile after the one on its way
    if (tid == 0) {
        const KdMeta m0 = kd_meta(p, t_begin, n_tiles, K);
        s_meta[0] = m0;
        kd_issue(p, m0, s_buf, &s_bar[0], kSym);
        if (t_begin + 1 < t_end) nx = kd_meta(p, t_begin + 1, n_tiles, K);
    }
    __syncthreads();
    {
        const KdMeta m = s_meta[0];
        const int nw = (n_rec - m.rb < kKRW) ? (int)(n_rec - m.rb) : kKRW;
        if (tid <= nw) {
            s_wp[0][tid] = p.wpre[m.rb + tid];
            s_sr[0][tid] = p.so[m.rb + tid];
        }
        if (!kd_wait(&s_bar[0], phase[0])) failed = true;
        phase[0] ^= 1u;
        kd_digitize(s_buf, (int)((p.head_pad + m.jlo) & 15), kd_nsym(m, K), tid, low);
    }
    __syncthreads();

    int b = 0;
    for (long long tile = t_begin; tile < t_end; ++tile, b ^= 1) {
        const bool more = tile + 1 < t_end;
        uint8_t *cur = s_buf + b * kSym;
        uint8_t *nxt = s_buf + (b ^ 1) * kSym;
        if (more && tid == 0) {  // the next tile's bytes on their way
            s_meta[b ^ 1] = nx;
            kd_issue(p, nx, nxt, &s_bar[b ^ 1], kSym);
            if (tile + 2 < t_end) nx = kd_meta(p, tile + 2, n_tiles, K);
        }
        const KdMeta m = s_meta[b];
        const long long w0 = tile * kKW;
        const long long w1 = (w0 + kKW < n_win) ? w0 + kKW : n_win;
        const long long rb = m.rb, jlo = m.jlo;
        const int nw = (n_rec - rb < kKRW) ? (int)(n_rec - rb) : kKRW;
        const long long *wp = s_wp[b], *sr = s_sr[b];
        const long long nsym = kd_nsym(m, K);
        const int lead = (int)((p.head_pad + jlo) & 15);
        const uint8_t *t_sym = cur + lead;  // t_sym[x] = digit of byte jlo + x

        // this thread's windows: entries and counts
        const long long wt = w0 + (long long)tid * kKPer;
        // more records start in this tile than the shared window holds: the
        // per-window path (searches past the window)
        const bool dense = rb + nw < n_rec && wp[nw] < w1;
        E e[kKPer];
        int sum = 0;
        bool vec = false;  // the eight entries are in e[] (else written one by one)
        if (!dense && wt < w1) {
            KCursor c = kc_init<K>(wt, nw, wp, sr, jlo);
            if (wt + kKPer <= w1 && c.rem >= kKPer * K && c.j >= 0 && c.j + kKPer * K <= nsym) {
                // all eight windows whole and in one record
                int ent[kKPer], cn[kKPer], ix[kKPer];
                ktab_fast_windows<K, T16>(cur, lead + c.j, p.klut, s_tab, ent, cn, ix);
#pragma unroll
                for (int q = 0; q < kKPer; ++q) {
                    sum += cn[q];
                    e[q] = ent[q] >= 0 ? KdEnt<E, K>::id(ent[q]) : KdEnt<E, K>::whole(ix[q]);
                }
                vec = true;
            } else {
                const int nq = (int)(w1 - wt < kKPer ? w1 - wt : kKPer);
                for (int q = 0; q < nq; ++q) {
                    const KWin a = kc_window<K, T16>(c, nw, rb, sr, jlo, t_sym, nsym, p.klut, s_tab);
                    sum += a.cnt;
                    went[wt + q] = kd_entry<E, K>(a, t_sym);
                }
            }
        } else if (dense) {
            int i = 0;
            for (int q = 0; q < kKPer; ++q) {
                const long long w = wt + q;
                if (w >= w1) break;
                const KWin a = ktab_window<K, T16>(w, i, nw, rb, n_rec, wp, sr, p.wpre, p.so, t_sym,
                                                   jlo, nsym, p.klut, s_tab);
                sum += a.cnt;
                went[w] = kd_entry<E, K>(a, t_sym);
            }
        }
        if (vec) kd_store_ents(went + wt, e);
        int x = sum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_wsum[warp] = x;
        __syncthreads();
        if (tid == 0) {
            long long total = 0;
#pragma unroll
            for (int w = 0; w < kKThreads / 32; ++w) total += s_wsum[w];
            p.tsum[tile] = total;
        }
        if (more) {
            // the next tile: its record window, then its digits once its bytes land
            const KdMeta mn = s_meta[b ^ 1];
            const int nn = (n_rec - mn.rb < kKRW) ? (int)(n_rec - mn.rb) : kKRW;
            if (tid <= nn) {
                s_wp[b ^ 1][tid] = p.wpre[mn.rb + tid];
                s_sr[b ^ 1][tid] = p.so[mn.rb + tid];
            }
            if (!kd_wait(&s_bar[b ^ 1], phase[b ^ 1])) failed = true;
            phase[b ^ 1] ^= 1u;
            kd_digitize(nxt, (int)((p.head_pad + mn.jlo) & 15), kd_nsym(mn, K), tid, low);
        }
        __syncthreads();  // the next tile is staged; this one's buffers are free
    }
    // (every copy issued has been waited for above, bounded)
    if (failed) set_dev_status(p.status, DEV_TIMEOUT);
    if (__syncthreads_or(low) && tid == 0) {
        if (*(volatile unsigned *)p.gate != p.epoch) *(volatile unsigned *)p.gate = p.epoch;
    }
}

// Entry q of a thread's entries, by selects (q not known at compile time).
template <typename E>
__device__ __forceinline__ E kd_pick(const E (&e)[kKPer], int q) {
    E r = e[0];
#pragma unroll
    for (int j = 1; j < kKPer; ++j)
        if (q == j) r = e[j];
    return r;
}

// One window's ids from its entry at tile position pos: the id, or one
// single-symbol id per digit of the index the entry carries (the last digit
// lowest); into the staged tile (s_tok + shift) or straight to the output.
template <typename E, int K>
__device__ __forceinline__ void kd_expand_one(E e, int pos, bool staged, int *s_tok, int shift,
                                              int *out, long long tb, long long cap,
                                              const int *s_ids) {
    int v;
    bool is_id;
    const int c = KdEnt<E, K>::decode(e, v, is_id);
    if (is_id) {
        if (staged) s_tok[shift + pos] = v;
        else if (tb + pos < cap) out[tb + pos] = v;
        return;
    }
    for (int y = c - 1; y >= 0; --y) {
        const int id = s_ids[v % 5];
        v /= 5;
        if (staged) s_tok[shift + pos + y] = id;
        else if (tb + pos + y < cap) out[tb + pos + y] = id;
    }
}

// The expand pass: a contiguous run of tiles per CTA.  Per tile each thread
// loads its kKPer consecutive entries (one tile ahead) and counts their ids;
// a block scan gives every window its position from the tile's token
// offset; the entries and positions go to shared memory, and the ids are
// then written window by window with consecutive windows on consecutive
// threads (so the few windows that expand to single-symbol ids, which come
// in runs, spread over a warp's lanes instead of loading one lane), into a
// staged tile written out in aligned 16-byte stores.  Last, the offsets of
// the records that start in the tile.
template <int K, typename E>
__global__ void __launch_bounds__(kKThreads) kd_expand_kernel(const KdParams p) {
    __shared__ long long s_wp[kKRW + 1];  // window offsets of records rb .. rb + kKRW
    __shared__ int s_wsum[kKThreads / 32];
    __shared__ __align__(16) int s_tok[kKTok + 4];
    __shared__ __align__(16) uint16_t s_wpos[kKW];  // token position of each window in the tile
    __shared__ __align__(16) E s_ent[kKW];          // the tile's entries
    __shared__ int s_ids[5];                        // base_ids
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const E *went = static_cast<const E *>(p.went);
    if (tid < 5) s_ids[tid] = p.ids.b[tid];  // (read after the first tile's scan barrier)
    pdl_wait();  // the scan has finished and its writes are visible
    if (*(volatile const unsigned *)p.gate == p.epoch) return;  // the general path redoes it
    const long long n_rec = p.n_seq;
    const long long n_win = p.wpre[n_rec];
    const long long n_tiles = (n_win + kKW - 1) / kKW;
    const long long t_begin = (long long)blockIdx.x * n_tiles / gridDim.x;
    const long long t_end = (long long)(blockIdx.x + 1) * n_tiles / gridDim.x;
    if (t_begin >= t_end) return;

    // the first tile: entries, record, token offset, and (in registers until
    // the scan's barrier) the record window
    E e[kKPer];
    kd_load_ents(went + t_begin * kKW + tid * kKPer, e);
    long long rb = p.tile_rec[t_begin], tb = p.tsum[t_begin];
    long long rwp = 0;
    if (tid <= kKRW && rb + tid <= n_rec) rwp = p.wpre[rb + tid];

    for (long long tile = t_begin; tile < t_end; ++tile) {
        const bool more = tile + 1 < t_end;
        // the next tile's loads in flight while this one is expanded
        E ne[kKPer];
        long long nrb = 0, ntb = 0;
        if (more) {
            kd_load_ents(went + (tile + 1) * kKW + tid * kKPer, ne);
            nrb = p.tile_rec[tile + 1];
            ntb = p.tsum[tile + 1];
        }
        const long long w0 = tile * kKW;
        const int nwin = (int)((n_win - w0 < kKW) ? n_win - w0 : kKW);  // windows in the tile
        const int nw = (n_rec - rb < kKRW) ? (int)(n_rec - rb) : kKRW;
        const int q0 = tid * kKPer;
        const int nq = nwin - q0 < 0 ? 0 : (nwin - q0 < kKPer ? nwin - q0 : kKPer);
        int sum = 0;
        bool plain = nq == kKPer;  // the usual case: eight plain ids
#pragma unroll
        for (int q = 0; q < kKPer; ++q) plain = plain && KdEnt<E, K>::is_id(e[q]);
        if (plain) {
            sum = kKPer;
        } else {
            for (int q = 0; q < nq; ++q) sum += KdEnt<E, K>::count(kd_pick(e, q));
        }
        kd_store_ents(s_ent + q0, e);
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        if (tid <= kKRW) s_wp[tid] = rwp;  // (free since the last tile's final barrier)
        __syncthreads();
        int loc = x - sum, total = 0;
#pragma unroll
        for (int w = 0; w < kKThreads / 32; ++w) {
            if (w < warp) loc += s_wsum[w];
            total += s_wsum[w];
        }
        // every window's position in the tile
        if (plain) {
            uint4 wp4;
            wp4.x = (unsigned)loc | ((unsigned)(loc + 1) << 16);
            wp4.y = (unsigned)(loc + 2) | ((unsigned)(loc + 3) << 16);
            wp4.z = (unsigned)(loc + 4) | ((unsigned)(loc + 5) << 16);
            wp4.w = (unsigned)(loc + 6) | ((unsigned)(loc + 7) << 16);
            *reinterpret_cast<uint4 *>(s_wpos + q0) = wp4;
        } else {
            for (int q = 0; q < nq; ++q) {
                s_wpos[q0 + q] = (uint16_t)loc;
                loc += KdEnt<E, K>::count(kd_pick(e, q));
            }
        }
        // staged: ids go to s_tok[shift + pos], shift being the misalignment
        // (in ids) of the tile's first output
        const int shift = (int)((reinterpret_cast<uintptr_t>(p.out + tb) >> 2) & 3u);
        const bool staged = total + shift <= kKTok;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kKPer; ++q) {
            const int w = q * kKThreads + tid;
            if (w < nwin) {
                const E ew = s_ent[w];
                const int pos = s_wpos[w];
                if (KdEnt<E, K>::is_id(ew) && staged) s_tok[shift + pos] = (int)ew;
                else kd_expand_one<E, K>(ew, pos, staged, s_tok, shift, p.out, tb, p.ids_cap, s_ids);
            }
        }
        __syncthreads();
        if (staged) {
            const int span = shift + total;
            int *g = p.out + (tb - shift);                  // 16-byte aligned
            const long long lim = p.ids_cap - (tb - shift);  // ids of g inside the buffer
            for (int q = tid; q < (span + 3) >> 2; q += kKThreads) {
                const int lo = q * 4, hi = lo + 4;
                if (lo >= shift && hi <= span && hi <= lim) {
                    *reinterpret_cast<int4 *>(g + lo) = *reinterpret_cast<const int4 *>(s_tok + lo);
                } else {
                    for (int y = lo > shift ? lo : shift; y < (hi < span ? hi : span); ++y)
                        if (y < lim) g[y] = s_tok[y];
                }
            }
        }
        // offsets of the records whose first window (or, empty, whose next
        // record's first window) is in this tile: record rb when it starts
        // here, and every later record that starts before the tile's end
        // (from the shared window, or from wpre when more start here than it
        // holds)
        const long long w1 = w0 + nwin;
        if (tid == 0 && s_wp[0] == w0) {
            long long r = rb;
            p.id_offsets[r] = tb;
            while (r > 0 && p.wpre[r - 1] == w0) p.id_offsets[--r] = tb;
        }
        const bool dense = rb + nw < n_rec && s_wp[nw] < w1;
        for (long long r = rb + 1 + tid; r <= (dense ? n_rec : rb + nw); r += kKThreads) {
            const long long w = (r - rb <= nw) ? s_wp[r - rb] : p.wpre[r];
            if (w >= w1) break;
            p.id_offsets[r] = tb + s_wpos[w - w0];
        }
        __syncthreads();  // s_tok, s_wpos, s_ent and the record window are free
        if (more) {
#pragma unroll
            for (int q = 0; q < kKPer; ++q) e[q] = ne[q];
            rb = nrb;
            tb = ntb;
            rwp = (tid <= kKRW && rb + tid <= n_rec) ? p.wpre[rb + tid] : 0;
        }
    }
}

template <int K, bool T16>
constexpr int kd_count_smem() {
    return ktab_tab_bytes(K, T16) + 2 * ktab_sym_bytes(K);
}

// Resident CTAs per SM of a count instantiation; the first call also raises
// its dynamic shared memory limit (dnatok_reserve makes that call, so a
// first encode under stream capture finds it done).
template <int K, bool T16, typename E>
cudaError_t kd_count_init(int *per_sm_out) {
    constexpr int smem = kd_count_smem<K, T16>();
    static std::atomic<int> per_sm{0};
    if (per_sm.load() == 0) {
        cudaError_t e = cudaFuncSetAttribute(kd_count_kernel<K, T16, E>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kd_count_kernel<K, T16, E>, kKThreads,
                                                          smem);
        if (e != cudaSuccess) return e;
        per_sm.store(n > 0 ? n : 1);
    }
    *per_sm_out = per_sm.load();
    return cudaSuccess;
}

template <int K, typename E>
int kd_expand_occupancy() {
    static std::atomic<int> per_sm{0};
    if (per_sm.load() == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kd_expand_kernel<K, E>, kKThreads, 0) !=
                cudaSuccess || n < 1)
            n = 1;
        per_sm.store(n);
    }
    return per_sm.load();
}

// Programmatic dependent launch: the CTAs start (and the count's load its
// table) while the kernel before them runs; they wait for it on the device.
template <typename Kern>
cudaError_t kd_launch_pdl(Kern kern, long long grid, int smem, const KdParams &p, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(grid < 1 ? 1 : grid));
    cfg.blockDim = dim3(kKThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

// One count or expand launch (with p.tile_rec null: only the count's setup).
template <int K, bool T16, typename E>
cudaError_t kd_launch(bool expand, const KdParams &p, int sm_count, long long max_tiles,
                      cudaStream_t s) {
    if (expand) {
        long long grid = (long long)sm_count * kd_expand_occupancy<K, E>();
        if (grid > max_tiles) grid = max_tiles;
        return kd_launch_pdl(kd_expand_kernel<K, E>, grid, 0, p, s);
    }
    int per_sm = 0;
    cudaError_t e = kd_count_init<K, T16, E>(&per_sm);
    if (e != cudaSuccess || !p.tile_rec) return e;
    long long grid = (long long)sm_count * per_sm;
    if (grid > max_tiles) grid = max_tiles;
    return kd_launch_pdl(kd_count_kernel<K, T16, E>, grid, kd_count_smem<K, T16>(), p, s);
}

cudaError_t kd_dispatch(int k, bool expand, bool t16, bool e16, const KdParams &p, int sm_count,
                        long long max_tiles, cudaStream_t s) {
#define DNATOK_KD_E(KK, TT)                                                                \
    if (e16) return kd_launch<KK, TT, uint16_t>(expand, p, sm_count, max_tiles, s);        \
    return kd_launch<KK, TT, int>(expand, p, sm_count, max_tiles, s);
#define DNATOK_KD_K(KK)                          \
    case KK:                                     \
        if (t16 && KK <= 6) {                    \
            DNATOK_KD_E(KK, (KK <= 6))           \
        } else {                                 \
            DNATOK_KD_E(KK, false)               \
        }
    switch (k) {
        DNATOK_KD_K(1) DNATOK_KD_K(2) DNATOK_KD_K(3) DNATOK_KD_K(4) DNATOK_KD_K(5)
        DNATOK_KD_K(6) DNATOK_KD_K(7) DNATOK_KD_K(8) DNATOK_KD_K(9) DNATOK_KD_K(10)
        default: return cudaErrorInvalidValue;
    }
#undef DNATOK_KD_K
#undef DNATOK_KD_E
}

}  // namespace

long long ktab_direct_tiles(long long n_bytes) { return n_bytes / kKW + 2; }

long long ktab_direct_entries(long long n_bytes, long long n_seq, int k) {
    // windows: sum of ceil(L / k) <= n / k + n_seq, whole tiles, one spare
    return ((n_bytes / k + n_seq) / kKW + 2) * (long long)kKW;
}

cudaError_t ktab_direct_setup(dnatok_handle *h) {
    KdParams none;
    std::memset(&none, 0, sizeof(none));
    return kd_dispatch(h->k, false, h->d_klut16 != nullptr, h->kent16, none, 1, 1, nullptr);
}

cudaError_t ktab_direct_launch(dnatok_handle *h, const uint8_t *bytes, long long n,
                               const long long *so, long long n_seq, long long *wpre,
                               long long *tile_rec, long long *tsum, void *went, int32_t *out,
                               long long ids_cap, long long *id_offsets, long long *totals,
                               unsigned epoch, cudaStream_t s) {
    const long long max_tiles = ktab_direct_tiles(n);
    // 1. window offsets and the tile map (one block)
    cudaError_t e = launch_window_plan(so, n_seq, n, h->k, wpre, tile_rec, max_tiles, kKWShift,
                                       h->d_gate, epoch, s);
    if (e != cudaSuccess) return e;
    KdParams p;
    std::memset(&p, 0, sizeof(p));
    p.head_pad = (int)((uintptr_t)bytes & 15u);
    p.base = bytes - p.head_pad;
    p.n = n;
    p.so = so;
    p.n_seq = n_seq;
    p.wpre = wpre;
    p.tile_rec = tile_rec;
    p.tsum = tsum;
    p.went = went;
    p.klut = h->d_klut;
    p.klut16 = h->d_klut16;
    for (int d = 0; d < 5; ++d) p.ids.b[d] = h->base_ids[d];
    p.out = out;
    p.ids_cap = ids_cap;
    p.id_offsets = id_offsets;
    p.gate = h->d_gate;
    p.epoch = epoch;
    p.status = h->d_status;
    const bool t16 = h->d_klut16 != nullptr;
    // 2. window entries and token counts per tile
    e = kd_dispatch(h->k, false, t16, h->kent16, p, h->sm_count, max_tiles, s);
    if (e != cudaSuccess) return e;
    // 3. tile offsets, totals, records with no window left
    // (skipped when the gate is up: a plan that declined left wpre unwritten)
    tile_scan_kernel<<<1, kTileScanThreads, 0, s>>>(tsum, nullptr, wpre, nullptr, n_seq, nullptr,
                                                    -1, kKW, id_offsets, totals, h->d_status,
                                                    h->d_gate, epoch, false);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // 4. ids and record offsets
    return kd_dispatch(h->k, true, t16, h->kent16, p, h->sm_count, max_tiles, s);
}

}  // namespace dnatok
