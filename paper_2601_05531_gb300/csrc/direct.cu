// direct.cu -- the direct path for RAW input without separators.
//
// When no byte of the input is a separator (or any other byte below 0x21),
// every byte is a kept symbol, so each record's token count is known from
// its length alone (ceil(L / k) k-mers with the tail UNK; L single-nucleotide
// ids or symbols), and every token's position in the output follows from the
// record offsets without looking at the data: token m of record r goes to
// id_offsets[r] + m.  Then the whole encode is embarrassingly parallel --
// no scan across tiles, no look-back:
//   1. direct_plan_kernel (one block) validates seq_offsets and writes
//      id_offsets and totals from the record lengths;
//   2. direct_kernel streams 16 KiB tiles (16-byte loads, SWAR classification
//      as in the tile kernel), writes the ids, and flags the launch when it
//      meets a byte below 0x21;
//   3. the general tile kernel is launched behind it gated on that flag: it
//      runs (and rewrites every output) only when the direct path's premise
//      failed, and exits at once otherwise.
// Paper: Algorithm 2's byte -> id gather and MapKmer, with the k-mer id in
// closed form sum_i 4^(k-1-i) * code(b_i) (Sec. 2.2).
#include <cstring>

#include "handle.h"
#include "tile_kernel.cuh"

namespace dnatok {

namespace {

constexpr int kDThreads = 256;
constexpr int kPlanThreads = 1024;
constexpr int kPlanTile = 4096;  // records per pass of the plan kernel

struct DirectParams {
    const uint8_t *base;       // bytes rounded down to 16
    int head_pad;              // bytes - base
    long long n;               // input bytes
    const long long *so;       // seq_offsets (n_seq + 1)
    long long n_seq;
    void *out;                 // int32 ids or uint8 symbols
    long long *offsets_out;    // id offsets (n_seq + 1)
    long long *totals_out;     // or null
    unsigned *gate;            // set to `epoch` when the general path must run
    unsigned epoch;
    int k;
    unsigned long long kinv;   // ceil(2^64 / k) for k >= 2: floor(x / k) = umulhi(x, kinv)
    const int *lut;            // MODE_CHAR
    long long n_tiles;
    // non-null (compacted FASTA): {n, n_seq, start, id base} are read here
    // on the device, written by kernels that finished before these start;
    // the input then begins `start` bytes after `base` (16-byte aligned) and
    // n and n_seq above are upper bounds (the grid is sized by n)
    const long long *dyn;
    long long d_base;          // output index of the first record's first id
    long long out_cap;         // ids capacity (the plan sends a larger encode to the general path)
    // table-driven k-mers (non-null only there): the plan also maps every
    // tile of 2^tile_shift windows to the record holding its first window
    long long *tile_rec;
    long long tile_cap;        // entries of tile_rec
    int tile_shift;
};

// The parameters with the device-side counts in place, or null when an
// earlier kernel of this encode already sent it to the general path.
__device__ __forceinline__ bool resolve_counts(DirectParams &q) {
    if (!q.dyn) return true;
    if (*(volatile const unsigned *)q.gate == q.epoch) return false;
    q.n = q.dyn[0];
    q.n_seq = q.dyn[1];
    const long long start = q.dyn[2];
    q.base += start & ~15ll;
    q.head_pad = (int)(start & 15);
    q.d_base = q.dyn[3];
    return q.n_seq >= 1;
}

// tokens of a record of L kept symbols: ceil(L / k) (L when k = 1)
__device__ __forceinline__ long long rec_tokens(const DirectParams &q, long long L) {
    return q.k == 1 ? L : (long long)__umul64hi((unsigned long long)(L + q.k - 1), q.kinv);
}

__device__ __forceinline__ void raise_gate(const DirectParams &q) {
    if (*(volatile unsigned *)q.gate != q.epoch) *(volatile unsigned *)q.gate = q.epoch;
}

// id offsets from the record lengths; any malformed offset sends the encode
// to the general path (which reports it).  One block (the direct kernel's
// CTAs start while it runs): passes of kPlanTile records, each loaded and
// stored coalesced through shared memory, one pass for up to 4096 records.
__global__ void __launch_bounds__(kPlanThreads) direct_plan_kernel(DirectParams q0) {
    constexpr int kPer = kPlanTile / kPlanThreads;
    __shared__ long long s_v[kPlanTile + 1];
    __shared__ long long wsum[kPlanThreads / 32];
    pdl_launch_dependents();  // the direct kernel may start loading its input now
    DirectParams q = q0;
    if (!resolve_counts(q)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = q.n_seq;
    bool bad = false;
    long long carry = q.d_base;  // output index of the first id of this pass
    for (long long r0 = 0; r0 < n; r0 += kPlanTile) {
        const int cnt = (n - r0 < kPlanTile) ? (int)(n - r0) : kPlanTile;
        {
            // every load of the pass in flight at once
            constexpr int kLd = (kPlanTile + 1 + kPlanThreads - 1) / kPlanThreads;
            long long v[kLd];
#pragma unroll
            for (int it = 0; it < kLd; ++it) {
                const int i = tid + it * kPlanThreads;
                v[it] = (i <= cnt) ? __ldg(q.so + r0 + i) : 0;
            }
#pragma unroll
            for (int it = 0; it < kLd; ++it) {
                const int i = tid + it * kPlanThreads;
                if (i <= cnt) s_v[i] = v[it];
            }
        }
        __syncthreads();
        // the list's two ends, from the staged offsets (no second round trip)
        if (tid == 0 && r0 == 0 && s_v[0] != 0) bad = true;
        if (tid == 0 && r0 + cnt == n && s_v[cnt] != q.n) bad = true;
        long long t[kPer], sum = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int i = tid * kPer + j;
            t[j] = 0;
            if (i < cnt) {
                const long long L = s_v[i + 1] - s_v[i];
                if (L < 0) bad = true;
                t[j] = rec_tokens(q, L);
                sum += t[j];
            }
        }
        long long x = sum;  // inclusive scan over the block
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();  // every s_v read above is done, wsum is complete
        long long pre = carry, tot = 0;
#pragma unroll
        for (int w = 0; w < kPlanThreads / 32; ++w) {
            if (w < warp) pre += wsum[w];
            tot += wsum[w];
        }
        long long run = pre + x - sum;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            s_v[tid * kPer + j] = run;
            run += t[j];
        }
        __syncthreads();
        if (q.tile_rec) {
            // the tiles whose first window lies in this pass's records, one
            // thread per tile: its record by a search of the staged window
            // offsets (at most tile_cap tiles, whatever the offsets hold)
            const int sh = q.tile_shift;
            const long long a = carry - q.d_base, b = a + tot;
            for (long long tt = ((a + (1ll << sh) - 1) >> sh) + tid; tt < q.tile_cap && (tt << sh) < b;
                 tt += kPlanThreads) {
                const long long w = (tt << sh) + q.d_base;
                int lo = 0, hi = cnt - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_v[mid] <= w) lo = mid; else hi = mid - 1;
                }
                q.tile_rec[tt] = r0 + lo;
            }
        }
        for (int i = tid; i < cnt; i += kPlanThreads) q.offsets_out[r0 + i] = s_v[i];
        carry += tot;
        __syncthreads();  // s_v and wsum are reused by the next pass
    }
    if (tid == 0 && (n == 0 || carry > q.out_cap)) bad = true;
    if (__syncthreads_or(bad)) {
        if (tid == 0) raise_gate(q);
        return;
    }
    if (tid == 0) {
        q.offsets_out[n] = carry;
        if (q.totals_out) {
            q.totals_out[0] = carry;
            q.totals_out[1] = n;
        }
    }
}

__device__ __forceinline__ unsigned dcodes4(unsigned x) { return ((x >> 1) ^ (x >> 2)) & 0x03030303u; }
__device__ __forceinline__ unsigned dnonbase4(unsigned x, unsigned c) {
    const unsigned t = c | (c >> 4);
    const unsigned sel = __byte_perm(t, 0, 0x0020);
    const unsigned u = __byte_perm(0x54474341u, 0, sel);
    const unsigned d = (x & 0xDFDFDFDFu) ^ u;
    return (((d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | d) & 0x80808080u;
}
__device__ __forceinline__ unsigned dlow4(unsigned x) {
    return ~((x | 0x80808080u) - 0x21212121u) & ~x & 0x80808080u;
}
__device__ __forceinline__ unsigned dgather4(unsigned m) {
    return (((m >> 7) & 0x01010101u) * 0x01020408u) >> 24;
}
// mask of the byte lanes of a vector at aligned position ab that lie in
// [lo, hi) (aligned coordinates), byte j in bit j
__device__ __forceinline__ unsigned lane_mask16(long long ab, long long lo, long long hi) {
    unsigned m = 0xFFFFu;
    if (ab < lo) m &= 0xFFFFu << (unsigned)(lo - ab < 16 ? lo - ab : 16);
    if (ab + 16 > hi) {
        const long long keep = hi - ab;
        m &= keep <= 0 ? 0u : ((1u << keep) - 1u);
    }
    return m & 0xFFFFu;
}

// Four byte-lane codes (0..3 in each lane's low bits) -> 8 bits in the top
// byte of the product, first byte in the two top bits: lane i's code lands at
// bit 30 - 2i; every other partial product falls outside bits 24..31 and no
// two land on the same bits, so nothing carries into them.
__device__ __forceinline__ unsigned pack4_hi(unsigned c) { return c * 0x40100401u; }

// One 16-byte vector: 2-bit codes (first byte in the top bits), N flags and
// below-0x21 flags (byte j in bit j).
struct Vec16 {
    unsigned codes, nflags, low;
};
__device__ __forceinline__ Vec16 classify16(const uint4 &w) {
    const unsigned c0 = dcodes4(w.x), c1 = dcodes4(w.y), c2 = dcodes4(w.z), c3 = dcodes4(w.w);
    Vec16 r;
    r.codes = (pack4_hi(c0) & 0xFF000000u) | ((pack4_hi(c1) >> 8) & 0x00FF0000u) |
              ((pack4_hi(c2) >> 16) & 0x0000FF00u) | (pack4_hi(c3) >> 24);
    // the letter each lane's code stands for, against the byte folded to
    // upper case: a difference anywhere means an N-class byte (and any byte
    // below 0x21 is one of those)
    auto diff = [](unsigned x, unsigned c) -> unsigned {
        const unsigned t = c | (c >> 4);
        const unsigned u = __byte_perm(0x54474341u, 0, __byte_perm(t, 0, 0x0020));
        return (x & 0xDFDFDFDFu) ^ u;
    };
    const unsigned d0 = diff(w.x, c0), d1 = diff(w.y, c1), d2 = diff(w.z, c2), d3 = diff(w.w, c3);
    r.nflags = 0u;
    r.low = 0u;
    if (d0 | d1 | d2 | d3) {  // rare: an N-class byte somewhere in the vector
        auto nz = [](unsigned d) -> unsigned {
            return (((d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | d) & 0x80808080u;
        };
        r.nflags = dgather4(nz(d0)) | (dgather4(nz(d1)) << 4) | (dgather4(nz(d2)) << 8) |
                   (dgather4(nz(d3)) << 12);
        r.low = dgather4(dlow4(w.x)) | (dgather4(dlow4(w.y)) << 4) | (dgather4(dlow4(w.z)) << 8) |
                (dgather4(dlow4(w.w)) << 12);
    }
    return r;
}

// Largest r in [0, n] with so[r] <= x (so[0] = 0 <= x), by one warp: 32-way
// probes narrow the range, so ~3 dependent rounds for 4096 records.
__device__ __forceinline__ long long warp_rec_search(const long long *so, long long n, long long x,
                                                     int lane) {
    long long lo = 0, hi = n;
    while (hi - lo > 31) {
        const long long step = ((hi - lo) >> 5) + 1;
        const long long idx = lo + lane * step;
        const bool ok = idx <= hi && so[idx] <= x;
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        const int L = 31 - __clz(b);
        const long long nlo = lo + L * step;
        if (L < 31 && nlo + step <= hi) hi = nlo + step - 1;
        lo = nlo;
    }
    const long long idx = lo + lane;
    const bool ok = idx <= hi && so[idx] <= x;
    const unsigned b = __ballot_sync(0xffffffffu, ok);
    return lo + (31 - __clz(b));
}

// ------------------------------------------------------------ k-mer ids
//
// Warp-streamed: each warp owns a contiguous run of 512-byte steps (one
// 16-byte vector per lane) and keeps kDepth steps in flight in registers.
// The k-mers that start in a lane's vector are written by that lane; the
// codes of the vector after it come from the next lane by shuffle (from the
// next step's lane 0 for lane 31, so a step is emitted one iteration after
// it is classified).  A step that lies inside one record (the usual case)
// needs only the warp-uniform phase of the record's k-mer frame and the
// output index of its next k-mer, both advanced in registers; steps that hold
// record boundaries resolve them per lane from a per-warp window of kWin
// entries of seq_offsets / id_offsets in shared memory.  No block-wide
// barrier anywhere.  k is a template parameter, so every shift, mask and
// division by k is a constant.

constexpr int kSThreads = 256;
constexpr int kSWarps = kSThreads / 32;
constexpr int kStep = 512;   // bytes per warp step
constexpr int kDepth = 4;    // warp steps in flight per lane
constexpr int kWin = 32;     // records in a warp's window

struct RecWin {
    long long s[kWin + 1];   // seq_offsets[rb .. rb + kWin] (n past the end)
    long long o[kWin];       // id_offsets[rb .. rb + kWin - 1]
};

// Largest r in [0, n] with so[r] <= x, by one warp (32-way probes).  Only
// reads so[0..n]; on non-monotone offsets it returns some index in range
// (the plan kernel rejects those before any result is used).
__device__ __forceinline__ long long warp_rec_search_safe(const long long *so, long long n,
                                                          long long x, int lane) {
    long long lo = 0, hi = n;
    for (int round = 0; round < 16 && hi - lo > 31; ++round) {
        const long long step = ((hi - lo) >> 5) + 1;
        const long long idx = lo + lane * step;
        const bool ok = idx <= hi && __ldg(so + idx) <= x;
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        if (b == 0u) return lo;
        const int L = 31 - __clz(b);
        const long long nlo = lo + L * step;
        if (L < 31 && nlo + step <= hi) hi = nlo + step - 1;
        lo = nlo;
    }
    const long long idx = lo + lane;
    const bool ok = idx <= hi && __ldg(so + idx) <= x;
    const unsigned b = __ballot_sync(0xffffffffu, ok);
    return b == 0u ? lo : lo + (31 - __clz(b));
}

// One 16-byte vector classified for the k-mer path: 2-bit codes (first byte
// in the top bits) and, when any byte is not one of ACGTacgt, the N flags
// (byte j in bit j) and the below-0x21 flags.
//
// A byte x is one of ACGTacgt iff its bits 0,3,4,6,7 are those of 'A' (0x41),
// or those of 'T' (0x50) when it is a T, T being bit 2 set and bit 1 clear:
// (x & 0xD9) ^ (0x41 + 0x0F * T) == 0.  The code is bit1^bit2 (low bit) and
// bit2^bit3 (high bit).
struct KVec {
    unsigned codes, bad;  // bad: nonzero iff a byte is not a base letter
};
__device__ __forceinline__ unsigned kv_word(unsigned x, unsigned &code) {
    const unsigned s1 = x >> 1, s2 = x >> 2;
    code = (s1 ^ s2) & 0x03030303u;
    const unsigned t = s2 & ~s1 & 0x01010101u;                 // T per byte
    return (x & 0xD9D9D9D9u) ^ (t * 0x0Fu + 0x41414141u);  // zero bytes: bases
}
__device__ __forceinline__ unsigned kv_pack(unsigned c0, unsigned c1, unsigned c2, unsigned c3) {
    // each product's top byte holds its word's four codes, first byte highest
    const unsigned p0 = c0 * 0x40100401u, p1 = c1 * 0x40100401u;
    const unsigned p2 = c2 * 0x40100401u, p3 = c3 * 0x40100401u;
    return __byte_perm(__byte_perm(p3, p2, 0x0073), __byte_perm(p1, p0, 0x0073), 0x5410);
}
// N flags of a vector from its four check words (zero byte = base), base i
// in bit i.  Two words' nonzero-byte flags go to bits 0 and 4 of each byte;
// one multiply then moves byte j's two flags to bits 24 + j and 28 + j (every
// partial product lands on its own bit, so nothing carries).
__device__ __forceinline__ unsigned kv_nflags(unsigned v0, unsigned v1, unsigned v2, unsigned v3) {
    auto nz = [](unsigned v) -> unsigned {  // 0x80 per nonzero byte
        return (((v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | v) & 0x80808080u;
    };
    const unsigned a = ((nz(v0) >> 7) | (nz(v1) >> 3)) * 0x01020408u;
    const unsigned b = ((nz(v2) >> 7) | (nz(v3) >> 3)) * 0x01020408u;
    return __byte_perm(a, b, 0x0073) & 0xFFFFu;  // bytes 2 and 3 of the permute are not zero
}

template <int K>
struct KC {
    static constexpr unsigned UNK = 1u << (2 * K);
    static constexpr unsigned KMASK = (1u << K) - 1u;
    static constexpr unsigned M32 = (unsigned)((0x100000000ull + K - 1) / K);  // ceil(2^32 / K)
    static constexpr int SLOTS = (16 + K - 1) / K;  // k-mer starts per vector, at most
    static constexpr int SURE = 16 / K;             // slots present whatever the phase
    static constexpr int PERW = 16 / K;             // k-mers per 16-base funnel window
    static constexpr int D = kStep % K;             // phase shift of a lane's next vector
    static constexpr int Q = kStep / K;             // k-mers it is ahead, less one on a wrap
    __device__ static __forceinline__ unsigned div(unsigned x) { return __umulhi(x, M32); }  // x < 2^17
};

// Record state of a warp between steps (all lanes hold the same values).
struct RecState {
    long long rb;   // record index of window entry 0
    long long obJ;  // output index of record ic's first k-mer starting at or after the step
    long long re;   // end of record ic
    int nv;         // records in the window: min(kWin, n_seq - rb)
    int ic;         // window index of the record holding the step's start
    int ph;         // that k-mer's start - the step's start (>= K only before the first byte)
    int give_up;    // more than kWin record starts in one step
};

// A step [X, X + kStep) that holds record boundaries, a record tail or the
// input's edges: every lane resolves its own records from the window, then
// the state moves on to the next step.
template <int K>
__device__ __forceinline__ RecState slow_step(RecState R, RecWin &W, const DirectParams &q, long long X,
                                           unsigned cw, unsigned cw_nx, unsigned nwin, bool advance) {
    using C = KC<K>;
    if (R.give_up) return R;  // the general path redoes everything
    const int lane = threadIdx.x & 31;
    const long long Xe = X + kStep;
    auto win_fill = [&](long long nrb) {
        __syncwarp();
        const long long i = nrb + lane;
        W.s[lane] = i <= q.n_seq ? __ldg(q.so + i) : q.n;
        if (lane == 0) W.s[kWin] = nrb + kWin <= q.n_seq ? __ldg(q.so + nrb + kWin) : q.n;
        W.o[lane] = i < q.n_seq ? q.offsets_out[i] : 0;
        R.rb = nrb;
        R.nv = (q.n_seq - nrb < kWin) ? (int)(q.n_seq - nrb) : kWin;
        __syncwarp();
    };
    // the window must hold every record that starts in [X, Xe)
    if (!(R.rb + R.nv >= q.n_seq || W.s[R.nv] >= Xe)) {
        if (R.ic > 0) {
            win_fill(R.rb + R.ic);
            R.ic = 0;
        }
        if (!(R.rb + R.nv >= q.n_seq || W.s[R.nv] >= Xe)) {
            R.give_up = 1;  // the general path takes over
            return R;
        }
    }
    auto kmer_at = [&](int o) -> unsigned {  // k-mer starting at byte o of the lane's vector
        const unsigned id = __funnelshift_l(cw_nx, cw, 2 * o) >> (32 - 2 * K);
        return ((nwin >> o) & C::KMASK) ? C::UNK : id;
    };
    int *const out = static_cast<int *>(q.out);
    const int x0r = 16 * lane;
    int i = R.ic;
    while (i + 1 < R.nv && W.s[i + 1] <= X + x0r) ++i;
    int p, rer;
    long long ob;
    if (i == R.ic) {
        const int qd = x0r > R.ph ? (int)C::div((unsigned)(x0r - R.ph + K - 1)) : 0;
        p = R.ph + qd * K;
        ob = R.obJ + qd;
    } else {
        const int rs = (int)(W.s[i] - X);
        const int qd = x0r > rs ? (int)C::div((unsigned)(x0r - rs + K - 1)) : 0;
        p = rs + qd * K;
        ob = W.o[i] + qd;
    }
    {
        const long long e = W.s[i + 1] - X;
        rer = e >= (1 << 30) ? (1 << 30) : (int)e;
    }
    {
        // the lane's record: k-mers at offsets o, o + K, ... below lim, the
        // same funnel windows as the fast path, tails to UNK
        const int o = p - x0r;  // >= 0
        const int lim = rer - x0r < 16 ? rer - x0r : 16;
        const int tail = rer - x0r - K;  // a k-mer at offset > tail runs past the record
        unsigned id[C::SLOTS];
#pragma unroll
        for (int t0 = 0; t0 < C::SLOTS; t0 += C::PERW) {
            const unsigned fw = __funnelshift_l(cw_nx, cw, 2 * (o + t0 * K));
#pragma unroll
            for (int t = t0; t < t0 + C::PERW && t < C::SLOTS; ++t)
                id[t] = __umulhi(fw << ((t - t0) * 2 * K), 1u << (2 * K));
        }
        int *dst = out + ob;
#pragma unroll
        for (int t = 0; t < C::SLOTS; ++t) {
            const int ot = o + t * K;
            if (ot < lim) {
                unsigned v = id[t];
                if (ot > tail || ((nwin >> ot) & C::KMASK)) v = C::UNK;
                dst[t] = (int)v;
            }
        }
    }
    if (rer < x0r + 16 && i + 1 < R.nv) {
        // rare: further records start inside this vector
        while (true) {
            ++i;
            p = rer;
            ob = W.o[i];
            const long long e = W.s[i + 1] - X;
            rer = e >= (1 << 30) ? (1 << 30) : (int)e;
            const int lim = rer < x0r + 16 ? rer : x0r + 16;
            int *dst = out + ob;
            for (int t = 0; p < lim; p += K, ++t) {
                const unsigned id = kmer_at(p - x0r);
                dst[t] = (int)(p + K > rer ? C::UNK : id);
            }
            if (rer >= x0r + 16 || i + 1 >= R.nv) break;
        }
    }
    if (!advance) return R;
    // the record state for the next step, which starts at Xe
    int j = R.ic;
    bool moved = false;
    while (true) {
        while (j + 1 < R.nv && W.s[j + 1] <= Xe) ++j;
        if (j + 1 == R.nv && R.rb + R.nv < q.n_seq && W.s[R.nv] <= Xe) {
            win_fill(R.rb + R.nv);  // slide past the window
            j = 0;
            moved = true;
            continue;
        }
        break;
    }
    if (j == R.ic && !moved) {
        // same record: its next k-mer start at or after Xe
        const int dd = R.ph - kStep;  // start - Xe
        if (dd < 0) {
            const unsigned qn = C::div((unsigned)(-dd + K - 1));
            R.ph = dd + (int)qn * K;
            R.obJ += qn;
        } else {
            R.ph = dd;
        }
    } else {  // a record that starts in (X, Xe]
        R.ic = j;
        const unsigned qn = C::div((unsigned)(Xe - W.s[j]) + K - 1);
        R.ph = (int)(W.s[j] + (long long)qn * K - Xe);
        R.obJ = W.o[j] + qn;
    }
    R.re = W.s[R.ic + 1];
    return R;
}

// 16-byte global -> shared copy that bypasses registers (zero-filled when
// `full` is false, in which case nothing is read)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool full) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem),
                 "r"(full ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The kernel's shape is tunable (dnatok_set_direct_launch, dnatok_autotune):
// kV 512-byte slots per warp step (one vector per lane each), and a ring of
// kRing steps per warp (kRing - 1 in flight); the supported pairs are the
// instantiations in launch_kmer_k.  Default: 2 slots, 4 steps.

// Classification of one 16-byte vector: packed codes and N flags.
struct KSlot {
    unsigned codes, nf;
};
__device__ __forceinline__ KSlot k_classify(const uint4 &w, bool real, long long ab, long long lo,
                                            long long hi, bool &sep) {
    unsigned c0, c1, c2, c3;
    const unsigned v0 = kv_word(w.x, c0), v1 = kv_word(w.y, c1);
    const unsigned v2 = kv_word(w.z, c2), v3 = kv_word(w.w, c3);
    KSlot r;
    r.codes = kv_pack(c0, c1, c2, c3);
    r.nf = 0u;
    if ((v0 | v1 | v2 | v3) != 0u) {  // rare: something other than a base letter
        r.nf = kv_nflags(v0, v1, v2, v3);
        if ((dlow4(w.x) | dlow4(w.y) | dlow4(w.z) | dlow4(w.w)) != 0u && real) {
            const unsigned low = dgather4(dlow4(w.x)) | (dgather4(dlow4(w.y)) << 4) |
                                 (dgather4(dlow4(w.z)) << 8) | (dgather4(dlow4(w.w)) << 12);
            if (low & lane_mask16(ab, lo, hi)) sep = true;
        }
    }
    return r;
}

template <int K, int kV, int kRing>
__global__ void __launch_bounds__(kSThreads, 4) direct_kmer_kernel(DirectParams q0) {
    static_assert(K >= 2 && K <= 15, "k-mer length");
    using C = KC<K>;
    constexpr int kSpan = kV * kStep;  // bytes per warp step
    // the gated general kernel behind this one may be scheduled as our CTAs
    // retire (it waits on the device for this grid to finish)
    pdl_launch_dependents();
    __shared__ RecWin wins[kSWarps];
    __shared__ uint4 ring_s[kSWarps][kRing][kV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RecWin &W = wins[warp];
    uint4 *const ring = &ring_s[warp][0][0][lane];  // this lane's slot 0 of stage 0
    // the steps are dealt out by the bound on n (the grid's size), then cut
    // at the data's end
    const long long S = (q0.head_pad + q0.n + kSpan - 1) / kSpan;
    DirectParams q = q0;
    if (!resolve_counts(q)) return;
    const long long lo = q.head_pad, hi = q.head_pad + q.n;  // valid aligned range
    const long long S_data = (hi + kSpan - 1) / kSpan;
    const long long nw = (long long)gridDim.x * kSWarps;
    const long long gw = (long long)blockIdx.x * kSWarps + warp;
    const long long s_begin = gw * S / nw;
    long long s_end = (gw + 1) * S / nw;
    if (s_end > S_data) s_end = S_data;
    if (s_begin >= s_end) return;
    const int n_steps = (int)(s_end - s_begin);

    // This lane's vectors: step u (relative to s_begin), slot v holds vector
    // (s_begin + u) * 64 + v * 32 + lane; step n_steps is the halo (its slot
    // 0, lane 0 only).
    const uint4 *const vp = reinterpret_cast<const uint4 *>(q.base) + s_begin * (kV * 32) + lane;
    int u_lim[kV];  // steps u < u_lim[v] are read by this lane in slot v
#pragma unroll
    for (int v = 0; v < kV; ++v) {
        const long long nvec = (hi + 15) / 16;  // vectors holding input bytes
        const long long mine = nvec - (s_begin * (kV * 32) + v * 32 + lane);
        const long long by_data = mine <= 0 ? 0 : (mine + kV * 32 - 1) / (kV * 32);
        const long long by_range = (v == 0 && lane == 0) ? n_steps + 1 : n_steps;
        u_lim[v] = (int)(by_data < by_range ? by_data : by_range);
    }
    const unsigned ring_sa = (unsigned)__cvta_generic_to_shared(ring);
    auto issue = [&](int u) {  // copy step u into its ring stage
        const unsigned sa = ring_sa + (unsigned)(u & (kRing - 1)) * (kV * 32 * 16);
        const uint4 *src = vp + (long long)u * (kV * 32);
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            // nothing is read when the size is zero (the slot is zero-filled)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa + v * 32 * 16),
                         "l"(src + v * 32), "r"(u < u_lim[v] ? 16 : 0)
                         : "memory");
        }
        cp_async_commit();
    };
#pragma unroll
    for (int u = 0; u < kRing - 1; ++u) issue(u);

    // The record holding the first step: seq_offsets is input, so this runs
    // while the plan kernel (a programmatic predecessor) is still working.
    const long long X0 = s_begin * kSpan - q.head_pad;
    RecState R;
    {
        long long r = warp_rec_search_safe(q.so, q.n_seq, X0 > 0 ? X0 : 0, lane);
        if (r > q.n_seq - 1) r = q.n_seq - 1;
        R.rb = r;
        R.ic = 0;
        R.give_up = 0;
        const long long i = r + lane;
        W.s[lane] = i <= q.n_seq ? __ldg(q.so + i) : q.n;
        if (lane == 0) W.s[kWin] = r + kWin <= q.n_seq ? __ldg(q.so + r + kWin) : q.n;
        R.nv = (q.n_seq - r < kWin) ? (int)(q.n_seq - r) : kWin;
    }
    // id offsets come from the plan kernel: wait for it, then see whether it
    // rejected seq_offsets
    pdl_wait();
    if (*(volatile const unsigned *)q.gate == q.epoch) {
        cp_async_wait<0>();
        return;
    }
    W.o[lane] = R.rb + lane < q.n_seq ? q.offsets_out[R.rb + lane] : 0;
    __syncwarp();
    {
        const long long xc = X0 > 0 ? X0 : 0, rs = W.s[0];
        const long long J = rec_tokens(q, xc - rs);  // ceil((xc - rs) / k)
        R.ph = (int)(rs + J * K - X0);
        R.obJ = W.o[0] + J;
        R.re = W.s[1];
    }

    // Warp-uniform fast-path state, in 32-bit coordinates relative to X0: the
    // 512-byte slot at Xr lies in one record (with 16 bytes to spare) iff
    // Xr <= lim.
    int Xr = 0, ph = R.ph;
    int *obp = static_cast<int *>(q.out) + R.obJ;  // out + output index of the next k-mer
    auto fast_lim = [&](long long re, long long X) -> int {
        if (X < 0) return -1;  // the head pad: the slow path
        const long long l = re - X0 - (kStep + 16);
        return l > (1 << 30) ? (1 << 30) : (l < -1 ? -1 : (int)l);
    };
    int lim = fast_lim(R.re, X0);
    const int c_lane = 16 * lane + K - 1;
    const int m32l = -32 * lane;

    // Per-lane fast-path state: a2 = 2 x the offset in the lane's vector of
    // its first k-mer start (in [0, 2K)), dp = that k-mer's output slot.
    // Rebuilt from the warp-uniform (ph, obp) of a slot starting at X; lane
    // 0's state is (2 ph, obp) again, which is how the slow path reads it.
    int a2;
    int *dp;
    auto lane_state = [&]() {
        const unsigned qd = C::div((unsigned)(c_lane - ph));
        a2 = 2 * ph + m32l + (int)qd * (2 * K);
        dp = obp + qd;
    };
    lane_state();
    bool synced = true;  // (ph, obp) hold the state of the next step (else lane 0 does)
    // k-mers of this lane's vector in a 512-byte slot inside a record; the
    // state then moves to the lane's vector of the next slot (512 bytes on)
    auto emit_fast = [&](unsigned cw, unsigned cw_nx, unsigned nwin, bool anyN) {
        unsigned id[C::SLOTS];
#pragma unroll
        for (int t0 = 0; t0 < C::SLOTS; t0 += C::PERW) {
            const unsigned fw = __funnelshift_l(cw_nx, cw, a2 + t0 * 2 * K);
#pragma unroll
            for (int t = t0; t < t0 + C::PERW && t < C::SLOTS; ++t)
                id[t] = __umulhi(fw << ((t - t0) * 2 * K), 1u << (2 * K));
        }
        if (anyN) {
#pragma unroll
            for (int t = 0; t < C::SLOTS; ++t)
                if ((nwin >> ((a2 >> 1) + t * K)) & C::KMASK) id[t] = C::UNK;
        }
#pragma unroll
        for (int t = 0; t < C::SLOTS; ++t)
            if (t < C::SURE || a2 + t * 2 * K < 32) dp[t] = (int)id[t];
        if (C::D == 0) {
            dp += C::Q;
        } else {
            const bool wrap = a2 < 2 * C::D;
            a2 += wrap ? 2 * (K - C::D) : -2 * C::D;
            dp += C::Q + (wrap ? 1 : 0);
        }
    };

    KSlot p[kV] = {};  // the previous step's slots
    bool sep = false, give_up = false;
    for (int u = 0; u <= n_steps; ++u) {
        issue(u + kRing - 1);
        cp_async_wait<kRing - 1>();  // step u has landed
        const uint4 *st = ring + (u & (kRing - 1)) * (kV * 32);
        KSlot c[kV];
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const long long ab = 16 * ((s_begin + u) * (kV * 32) + v * 32 + lane);
            c[v] = (v == 0 || u < n_steps) ? k_classify(st[v * 32], u < n_steps, ab, lo, hi, sep)
                                           : KSlot{0u, 0u};
        }
        if (u > 0) {
            // emit step u - 1 (slots p[]); a slot's lane 31 takes the next
            // slot's lane 0
            unsigned nx[kV];
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                const unsigned a = __shfl_down_sync(0xffffffffu, p[v].codes, 1);
                const unsigned b = __shfl_sync(0xffffffffu, v + 1 < kV ? p[v + 1].codes : c[0].codes, 0);
                nx[v] = lane == 31 ? b : a;
            }
            unsigned any = lane == 0 ? c[0].nf : 0u;
#pragma unroll
            for (int v = 0; v < kV; ++v) any |= p[v].nf;
            const bool anyN = __any_sync(0xffffffffu, any != 0u);
            unsigned nwin[kV];
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                nwin[v] = 0u;
                if (anyN) {
                    const unsigned a = __shfl_down_sync(0xffffffffu, p[v].nf, 1);
                    const unsigned b = __shfl_sync(0xffffffffu, v + 1 < kV ? p[v + 1].nf : c[0].nf, 0);
                    nwin[v] = p[v].nf | ((lane == 31 ? b : a) << 16);
                }
            }
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                if (Xr <= lim) {
                    emit_fast(p[v].codes, nx[v], nwin[v], anyN);
                    synced = false;
                } else {
                    // record boundaries, a tail or the input's edge in this slot
                    if (!synced) {  // the fast slots left the state in the lanes
                        ph = __shfl_sync(0xffffffffu, a2, 0) >> 1;
                        obp = reinterpret_cast<int *>(
                            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(dp), 0));
                    }
                    R.ph = ph;
                    R.obJ = obp - static_cast<int *>(q.out);
                    R = slow_step<K>(R, W, q, X0 + Xr, p[v].codes, nx[v], nwin[v],
                                     v + 1 < kV || u < n_steps);
                    ph = R.ph;
                    obp = static_cast<int *>(q.out) + R.obJ;
                    synced = true;
                    if (R.give_up) {
                        give_up = true;
                        lim = -(1 << 30);  // every later slot: slow_step, which returns at once
                    } else {
                        lim = fast_lim(R.re, X0 + Xr + kStep);
                        lane_state();
                    }
                }
                Xr += kStep;
            }
        }
#pragma unroll
        for (int v = 0; v < kV; ++v) p[v] = c[v];
    }
    cp_async_wait<0>();
    if (give_up) {
        if (lane == 0) raise_gate(q);
        return;
    }
    if (__any_sync(0xffffffffu, sep) && lane == 0) raise_gate(q);
}

// Single-nucleotide ids / BPE symbols: one output per byte at the byte's own
// position (no separators), streamed with 16-byte loads.
template <int MODE>
__global__ void __launch_bounds__(kDThreads) direct_byte_kernel(DirectParams q) {
    __shared__ int lut_s[256];
    const int tid = threadIdx.x;
    // one output per byte: the id offsets are seq_offsets itself, so this
    // kernel needs no plan -- it copies and validates them on the way (a
    // malformed list raises the flag; the general kernel then reports it)
    {
        bool bad = false;
        for (long long r = blockIdx.x * (long long)kDThreads + tid; r <= q.n_seq;
             r += (long long)gridDim.x * kDThreads) {
            const long long v = __ldg(q.so + r);
            q.offsets_out[r] = v;
            if (r < q.n_seq && __ldg(q.so + r + 1) < v) bad = true;
            if ((r == 0 && v != 0) || (r == q.n_seq && v != q.n)) bad = true;
        }
        if (bad) raise_gate(q);
        if (blockIdx.x == 0 && tid == 0 && q.totals_out) {
            q.totals_out[0] = q.n;
            q.totals_out[1] = q.n_seq;
        }
    }
    if (MODE == MODE_CHAR) {
        for (int i = tid; i < 256; i += kDThreads) lut_s[i] = q.lut[i];
        __syncthreads();
    }
    const long long lo = q.head_pad, hi = q.head_pad + q.n;
    bool sep = false;
    const long long n_vec = (hi + 15) / 16;
    for (long long vi = blockIdx.x * (long long)kDThreads + tid; vi < n_vec;
         vi += (long long)gridDim.x * kDThreads) {
        const long long ab = 16 * vi;
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(q.base + ab));
        const bool whole = (ab >= lo) && (ab + 16 <= hi);
        const unsigned m = whole ? 0xFFFFu : lane_mask16(ab, lo, hi);
        const long long x0 = ab - q.head_pad;
        const unsigned bw[4] = {w.x, w.y, w.z, w.w};
        if (dlow4(w.x) | dlow4(w.y) | dlow4(w.z) | dlow4(w.w)) {
            const unsigned l16 = dgather4(dlow4(w.x)) | (dgather4(dlow4(w.y)) << 4) |
                                 (dgather4(dlow4(w.z)) << 8) | (dgather4(dlow4(w.w)) << 12);
            if (l16 & m) sep = true;
        }
        if (MODE == MODE_SYM) {
            unsigned o[4];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const unsigned c = dcodes4(bw[g]);
                const unsigned n = dnonbase4(bw[g], c);  // 0x80 per N-class lane
                const unsigned nm = (n >> 7) * 0xFFu;    // 0xFF per N-class lane
                o[g] = (c & ~nm) | (0x04040404u & nm);
            }
            uint8_t *out = static_cast<uint8_t *>(q.out);
            if (whole && q.head_pad == 0) {
                *reinterpret_cast<uint4 *>(out + x0) = make_uint4(o[0], o[1], o[2], o[3]);
            } else {
                for (int j = 0; j < 16; ++j)
                    if ((m >> j) & 1u) out[x0 + j] = (uint8_t)(o[j >> 2] >> (8 * (j & 3)));
            }
        } else {
            int id[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) id[j] = lut_s[(bw[j >> 2] >> (8 * (j & 3))) & 0xFFu];
            int *out = static_cast<int *>(q.out);
            if (whole && q.head_pad == 0) {
                int4 *o4 = reinterpret_cast<int4 *>(out + x0);
                o4[0] = make_int4(id[0], id[1], id[2], id[3]);
                o4[1] = make_int4(id[4], id[5], id[6], id[7]);
                o4[2] = make_int4(id[8], id[9], id[10], id[11]);
                o4[3] = make_int4(id[12], id[13], id[14], id[15]);
            } else {
                for (int j = 0; j < 16; ++j)
                    if ((m >> j) & 1u) out[x0 + j] = id[j];
            }
        }
    }
    if (__syncthreads_or(sep) && tid == 0) raise_gate(q);
}

template <int KV, int KR>
cudaError_t launch_kmer_kv(int k, const cudaLaunchConfig_t &cfg, const DirectParams &q) {
    switch (k) {
#define DNATOK_K(KK) \
    case KK: return cudaLaunchKernelEx(&cfg, direct_kmer_kernel<KK, KV, KR>, q);
        DNATOK_K(2) DNATOK_K(3) DNATOK_K(4) DNATOK_K(5) DNATOK_K(6) DNATOK_K(7) DNATOK_K(8)
        DNATOK_K(9) DNATOK_K(10) DNATOK_K(11) DNATOK_K(12) DNATOK_K(13) DNATOK_K(14) DNATOK_K(15)
#undef DNATOK_K
        default: return cudaErrorInvalidValue;
    }
}

// resident CTAs per SM of one instantiation (the same for every k)
template <int KV, int KR>
int kmer_occupancy() {
    static int occ = 0;
    if (occ == 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, direct_kmer_kernel<6, KV, KR>, kSThreads,
                                                          0) != cudaSuccess || o < 1)
            o = 1;
        occ = o;
    }
    return occ;
}

}  // namespace

bool direct_eligible(int mode, long long n_seq, const int32_t *lut_host) {
    if (n_seq < 1 || n_seq > 65536) return false;
    if (mode == MODE_CHAR) {
        for (int b = 0x21; b < 256; ++b)
            if (lut_host[b] < 0) return false;  // the table drops a byte the direct path keeps
    }
    return mode == MODE_CHAR || mode == MODE_KMER || mode == MODE_SYM;
}

bool direct_shape_supported(const DirectShape &sh) {
    const bool pair = (sh.slots == 2 && sh.ring == 4) || (sh.slots == 1 && sh.ring == 8) ||
                      (sh.slots == 4 && sh.ring == 2);
    return pair && sh.ctas_per_sm >= 0 && sh.ctas_per_sm <= 4;
}

cudaError_t launch_direct(int mode, const uint8_t *bytes, long long n, const long long *so,
                          long long n_seq, void *out, long long *offsets_out,
                          long long *totals_out, unsigned *gate, unsigned epoch, int k,
                          const int *lut, int sm_count, const DirectShape &shape,
                          cudaStream_t s, const long long *dyn, long long out_cap,
                          cudaEvent_t ev0, cudaEvent_t ev1) {
    DirectParams q;
    q.tile_rec = nullptr;
    q.tile_cap = 0;
    q.tile_shift = 0;
    q.dyn = dyn;
    q.d_base = 0;
    q.out_cap = out_cap;
    q.head_pad = (int)((uintptr_t)bytes & 15u);
    q.base = bytes - q.head_pad;
    q.n = n;
    q.so = so;
    q.n_seq = n_seq;
    q.out = out;
    q.offsets_out = offsets_out;
    q.totals_out = totals_out;
    q.gate = gate;
    q.epoch = epoch;
    q.k = k;
    q.kinv = k > 1 ? ~0ull / (unsigned long long)k + 1ull : 0ull;
    q.lut = lut;
    q.n_tiles = 0;
    const bool kmer = mode == MODE_KMER && k >= 2;
    if (dyn && !kmer) return cudaErrorInvalidValue;  // device-side counts: k-mers only
    if (!kmer) {
        // single-nucleotide ids, symbols, and 1-mers (the default table maps
        // A/C/G/T to 0..3 and every other kept byte to 4 = UNK): one kernel,
        // no plan
        long long g2 = ((q.head_pad + n + 15) / 16 + kDThreads - 1) / kDThreads;
        const long long g3 = (n_seq + 1 + kDThreads - 1) / kDThreads;
        if (g2 < g3) g2 = g3;
        if (g2 > (long long)sm_count * 8) g2 = (long long)sm_count * 8;
        if (g2 < 1) g2 = 1;
        if (mode != MODE_SYM)
            direct_byte_kernel<MODE_CHAR><<<(unsigned)g2, kDThreads, 0, s>>>(q);
        else
            direct_byte_kernel<MODE_SYM><<<(unsigned)g2, kDThreads, 0, s>>>(q);
        return cudaGetLastError();
    }
    direct_plan_kernel<<<1, kPlanThreads, 0, s>>>(q);
    if (n > 0) {
        // programmatic dependent launch: it starts while the plan runs
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(kSThreads);
        cfg.stream = s;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr.val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        // one wave of resident CTAs (at most shape.ctas_per_sm per SM), every
        // warp with at least one step
        const int kv = shape.slots, kr = shape.ring;
        int occ = kv == 1 ? kmer_occupancy<1, 8>() : kv == 4 ? kmer_occupancy<4, 2>()
                                                            : kmer_occupancy<2, 4>();
        if (shape.ctas_per_sm > 0 && shape.ctas_per_sm < occ) occ = shape.ctas_per_sm;
        const long long steps = (q.head_pad + n + kv * kStep - 1) / (kv * kStep);
        long long grid = (long long)sm_count * occ;
        const long long need = (steps + kSWarps - 1) / kSWarps;
        if (grid > need) grid = need;
        cfg.gridDim = dim3((unsigned)grid);
        cudaError_t e = cudaSuccess;
        if (ev0) e = cudaEventRecord(ev0, s);  // timing: the kernel then waits for the plan
        if (e != cudaSuccess) return e;
        if (kv == 1 && kr == 8) e = launch_kmer_kv<1, 8>(k, cfg, q);
        else if (kv == 4 && kr == 2) e = launch_kmer_kv<4, 2>(k, cfg, q);
        else e = launch_kmer_kv<2, 4>(k, cfg, q);
        if (e == cudaSuccess && ev1) e = cudaEventRecord(ev1, s);
        return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_window_plan(const long long *so, long long n_seq, long long n, int k,
                               long long *wpre, long long *tile_rec, long long tile_cap,
                               int tile_shift, unsigned *gate, unsigned epoch, cudaStream_t s) {
    DirectParams q;
    std::memset(&q, 0, sizeof(q));
    q.n = n;
    q.so = so;
    q.n_seq = n_seq;
    q.offsets_out = wpre;
    q.gate = gate;
    q.epoch = epoch;
    q.k = k;
    q.kinv = k > 1 ? ~0ull / (unsigned long long)k + 1ull : 0ull;
    q.out_cap = 0x7fffffffffffffffll;
    q.tile_rec = tile_rec;
    q.tile_cap = tile_cap;
    q.tile_shift = tile_shift;
    direct_plan_kernel<<<1, kPlanThreads, 0, s>>>(q);
    return cudaGetLastError();
}

}  // namespace dnatok
