// ktab.cuh -- the shared pieces of the table-driven k-mer kernels (the
// two-pass kernels over the symbol plane and the count pass over raw
// bytes): tile constants, shared-memory sizing, and the per-window
// walk that turns k staged digits (A0 C1 G2 T3, 4 for N-class) into a
// base-5 table index and a token count (Algorithm 2, MapKmer).
#pragma once
#include <cstdint>

#include "common.cuh"

namespace dnatok {

// Largest r in [0, n_rec - 1] with srec[r] <= j (srec sorted, srec[0] = 0),
// by one thread.
__device__ __forceinline__ long long ovl_find(const long long *srec, long long n_rec, long long j) {
    long long lo = 0, hi = n_rec - 1;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (srec[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------ table-driven k-mers

constexpr int kKWShift = 11;
constexpr int kKW = 1 << kKWShift;  // windows per tile
constexpr int kKThreads = 256;
constexpr int kKPer = kKW / kKThreads;  // consecutive windows per thread
constexpr int kKRW = 64;        // records of a tile kept in shared memory
constexpr int kKTok = 2560;     // ids of a tile staged in shared memory by the emit

struct KtabIds {
    int b[5];  // ids of the single symbols A C G T N
};

__host__ __device__ constexpr int pow5(int k) { return k == 0 ? 1 : 5 * pow5(k - 1); }

// Dynamic shared memory of a ktab_tile_kernel: [u16 table (T16)] [symbols]
// [staged ids (EMIT)], each part 16-byte aligned.
__host__ __device__ constexpr int ktab_tab_bytes(int K, bool T16) {
    return T16 ? ((pow5(K) * 2 + 15) / 16) * 16 : 0;
}
__host__ __device__ constexpr int ktab_sym_bytes(int K) { return ((kKW * K + 32 + 15) / 16) * 16; }
__host__ __device__ constexpr int ktab_smem(int K, bool EMIT, bool T16) {
    return ktab_tab_bytes(K, T16) + ktab_sym_bytes(K) + (EMIT ? kKTok * 4 + 16 : 0);
}

// One window: its record (r, its first window wp, its symbol range [sr, sr1))
// from the tile's shared record window (advancing the caller's index i, as
// windows only grow), else by a search of wpre.
struct KWin {
    long long r, t, j;  // record, window within the record, first symbol in s_sym
    int cnt, ent;       // tokens; the table entry of a whole window (-1: none)
    int idx;            // a whole window's base-5 index
};

template <int K, bool T16>
__device__ __forceinline__ KWin ktab_window(long long w, int &i, int nw, long long rb, long long n_rec,
                                            const long long *s_wp, const long long *s_sr,
                                            const long long *wpre, const long long *srec,
                                            const uint8_t *s_sym, long long jlo, long long nsym,
                                            const int *klut, const uint16_t *s_tab) {
    KWin q;
    q.r = -1;
    q.cnt = 0;
    q.ent = -1;
    q.idx = 0;
    long long wp, sr, sr1;
    if (w >= s_wp[nw] && rb + nw < n_rec) {
        // more records start in this tile than the window holds
        const long long r = ovl_find(wpre, n_rec, w);
        q.r = r;
        wp = wpre[r];
        sr = srec[r];
        sr1 = srec[r + 1];
    } else {
        while (i + 1 < nw && s_wp[i + 1] <= w) ++i;
        q.r = rb + i;
        wp = s_wp[i];
        sr = s_sr[i];
        sr1 = s_sr[i + 1];
    }
    q.t = w - wp;
    q.j = sr + q.t * K - jlo;
    const long long rem = (sr1 - sr) - q.t * K;
    const int n_s = rem >= K ? K : (int)rem;
    if (q.j < 0 || n_s < 1 || q.j + n_s > nsym) {  // (malformed input)
        q.r = -1;
        return q;
    }
    if (n_s == K) {
        int index = 0;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            const int d = s_sym[q.j + x];
            index = index * 5 + (d < 5 ? d : 4);
        }
        if (T16) {
            const unsigned v = s_tab[index];
            q.ent = v == 0xFFFFu ? -1 : (int)v;
        } else {
            q.ent = __ldg(klut + index);
        }
        q.cnt = q.ent >= 0 ? 1 : K;
        q.idx = index;
    } else {
        q.cnt = n_s;
    }
    return q;
}

// A thread's walk over its consecutive windows in 32-bit tile-local terms:
// record i of the tile's shared window, j = the window's first symbol in the
// staged symbols, rem = symbols of the record from j on (clamped).  Set up
// once per thread; each window then costs a few int operations.
struct KCursor {
    int i, j, rem;
    bool first;  // the window is its record's first
};

template <int K>
__device__ __forceinline__ KCursor kc_init(long long w, int nw, const long long *s_wp,
                                           const long long *s_sr, long long jlo) {
    KCursor c;
    int i = 0;
    while (i + 1 < nw && s_wp[i + 1] <= w) ++i;
    const long long t = w - s_wp[i];
    const long long rem = (s_sr[i + 1] - s_sr[i]) - t * K;
    c.i = i;
    c.j = (int)(s_sr[i] + t * K - jlo);
    c.rem = (int)(rem < (1ll << 30) ? rem : (1ll << 30));
    c.first = (t == 0);
    return c;
}

// The window at the cursor (then advanced by one window), or cnt = 0 with
// r = -1 past the shared window's records or on malformed input.
template <int K, bool T16>
__device__ __forceinline__ KWin kc_window(KCursor &c, int nw, long long rb, const long long *s_sr,
                                          long long jlo, const uint8_t *s_sym, long long nsym,
                                          const int *klut, const uint16_t *s_tab) {
    KWin q;
    q.r = -1;
    q.cnt = 0;
    q.ent = -1;
    q.idx = 0;
    while (c.rem <= 0 && c.i + 1 < nw) {  // the record's windows are used up: the next record's
        ++c.i;
        const long long len = s_sr[c.i + 1] - s_sr[c.i];
        c.j = (int)(s_sr[c.i] - jlo);
        c.rem = (int)(len < (1ll << 30) ? len : (1ll << 30));
        c.first = true;
    }
    const int n_s = c.rem >= K ? K : c.rem;
    if (n_s < 1 || c.j < 0 || c.j + n_s > nsym) return q;  // (malformed input)
    q.r = rb + c.i;
    q.t = c.first ? 0 : 1;
    q.j = c.j;
    if (n_s == K) {
        int index = 0;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            const int d = s_sym[c.j + x];
            index = index * 5 + (d < 5 ? d : 4);
        }
        if (T16) {
            const unsigned v = s_tab[index];
            q.ent = v == 0xFFFFu ? -1 : (int)v;
        } else {
            q.ent = __ldg(klut + index);
        }
        q.cnt = q.ent >= 0 ? 1 : K;
        q.idx = index;
    } else {
        q.cnt = n_s;
    }
    c.j += K;
    c.rem -= K;
    c.first = false;
    return q;
}

// The kKPer whole windows of one record starting at staged symbol A (all in
// shared memory): the span is read as 32-bit words and shifted into place
// once, and each window's digits are then taken from registers at
// compile-time positions (instead of k single-byte shared-memory loads per
// window).  ent[q] = the table entry (-1: none), cnt[q] = 1 or K, idx[q] =
// the window's base-5 index.
template <int K, bool T16>
__device__ __forceinline__ void ktab_fast_windows(const uint8_t *s_base, int A, const int *klut,
                                                  const uint16_t *s_tab, int (&ent)[kKPer],
                                                  int (&cnt)[kKPer], int (&idx)[kKPer]) {
    constexpr int NB = kKPer * K;          // bytes of the span
    constexpr int NW = (NB + 3) / 4 + 1;   // words read (one more for the shift)
    const uint32_t *w32 = reinterpret_cast<const uint32_t *>(s_base + (A & ~3));
    const unsigned sh = 8u * (unsigned)(A & 3);
    uint32_t W[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) W[i] = w32[i];
    uint32_t X[NW - 1];
#pragma unroll
    for (int i = 0; i < NW - 1; ++i) X[i] = __funnelshift_r(W[i], W[i + 1], sh);
#pragma unroll
    for (int q = 0; q < kKPer; ++q) {
        int index = 0;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            const int b = q * K + x;
            const int d = (int)((X[b >> 2] >> (8 * (b & 3))) & 0xFFu);
            index = index * 5 + (d < 5 ? d : 4);
        }
        int e;
        if (T16) {
            const unsigned v = s_tab[index];
            e = v == 0xFFFFu ? -1 : (int)v;
        } else {
            e = __ldg(klut + index);
        }
        ent[q] = e;
        cnt[q] = e >= 0 ? 1 : K;
        idx[q] = index;
    }
}

}  // namespace dnatok
