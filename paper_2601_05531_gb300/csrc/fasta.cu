// fasta.cu -- FASTA text to compacted sequence bytes and record starts, the
// input of the direct k-mer kernel (reading C4: a line whose first byte is
// '>' is a header, dropped through its newline, and opens a record; bytes
// before the first header form a record only if byte 0 is not '>';
// '\n' '\r' ' ' '\t' are dropped everywhere).
//
// Line state.  Byte i starts a line when i = 0 or byte i-1 is '\n'; a line
// start holding '>' starts a header, which runs through the next '\n'.  A
// 16-byte vector is entered inside a header exactly when its byte 0 is not a
// line start and the last line start before it started a header.  So the
// only state carried along the text is the kind of the last line start (none,
// sequence, header): a "last one wins" scan of one small value per vector,
// followed by a sum scan of the vectors' kept-byte counts.  Inside a warp the
// first is two ballots (lanes with a line start, lanes whose last line start
// is a header).
//
// The text is cut into spans of 4 KiB, one warp each (8 rounds of 512 bytes,
// one 16-byte vector per lane per round), eight spans per CTA.  Three kernels:
//   fasta_sum_kernel   per span, entered outside a header: its kept bytes,
//                      the kept bytes before its first newline (the ones a
//                      span entered inside a header drops), its header lines
//                      and the kind of its last line start; the same for each
//                      CTA's eight spans in order;
//   fasta_scan_kernel  one block over the CTA summaries (coalesced through
//                      shared memory): every CTA's incoming state, kept offset
//                      and headers before it; the totals;
//   fasta_emit_kernel  per span: its incoming state (its CTA's, then the
//                      CTA's spans before it), each vector's by warp scans,
//                      its kept bytes packed and ORed into a per-warp
//                      shared-memory window aligned to the output's 16-byte
//                      grid, whole 16-byte pieces stored as vectors (the
//                      span's two partial ends byte by byte, as they are
//                      shared with the neighbouring spans), and the record
//                      starts.
#include "handle.h"

// Workspace of the compacted FASTA path, grown on demand (never under stream
// capture: dnatok_reserve sizes it beforehand).
struct FastaState {
    uint8_t *cbytes = nullptr;  // kept bytes (16-byte aligned, n + 64)
    long long cbytes_cap = 0;
    long long *cso = nullptr;   // record starts, then the kept total
    long long cso_cap = 0;
    uint4 *ssum = nullptr;      // per span: {kept, kept if entered in a header, headers, kind}
    long long spans_cap = 0;
    uint4 *csum = nullptr;      // per CTA (8 spans): the same
    longlong2 *sin = nullptr;   // per CTA: {kept offset, 2 * headers before + in header}
    long long ctas_cap = 0;
    long long *info = nullptr;  // kInfo words: counts for the direct kernels and the finish
    long long *plan = nullptr;  // per record (and the end): first id (stream chunks)
};

namespace dnatok {

namespace {

constexpr int kFWarps = 8;                    // warps per CTA
constexpr int kFT = 32 * kFWarps;             // threads per CTA
constexpr int kFRounds = 8;                   // 512-byte rounds per span
constexpr long long kFSpan = kFRounds * 512;  // bytes per span (one warp)
constexpr int kWinWords = 136;                // per-warp output window (544 bytes)
constexpr int kScanT = 1024;                  // threads of the scan kernel
constexpr long long kMaxRecords = 65536;      // records the direct kernel's plan takes
constexpr long long kFastaMin = 64 << 10;     // smallest input the compacted path takes
constexpr unsigned kFull = 0xffffffffu;

// The info words (device): the first four are the direct kernels' counts.
enum : int {
    I_N = 0,      // input bytes of the direct kernels (the open last record cut to whole k-mers)
    I_NREC = 1,   // records of the chunk (the continued one first)
    I_START = 2,  // where that input begins after the kept bytes' buffer: 16 - I_M
    I_DBASE = 3,  // output index of the first record's next id
    I_M = 4,      // symbols carried in front of the kept bytes (the continued record's partial k-mer)
    I_G0 = 5,     // global boundary index of the first record that starts here
    I_CONT = 6,   // 1 when the first record continues one from an earlier chunk
    I_END = 7,    // I_M + kept bytes
    I_HSTATE = 8, // line state after the chunk (HS_*)
    I_REC0 = 9,   // record index of the first header
    kInfo = 16
};
constexpr long long kHead = 16;  // kept bytes start this far into the buffer

// kinds of a line start (the scan's value; 0 = none)
enum : unsigned { LS_NONE = 0, LS_SEQ = 2, LS_HDR = 3 };

// 0x80 in every zero byte of t
__device__ __forceinline__ unsigned f_zero(unsigned t) {
    return ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u;
}
// 0x80 flags of a word -> bits 0..3
__device__ __forceinline__ unsigned f_bits4(unsigned f) {
    return (((f >> 7) & 0x01010101u) * 0x01020408u) >> 24;
}
// byte j of the vector equal to c -> bit j
__device__ __forceinline__ unsigned f_eq16(const uint4 &w, unsigned c) {
    const unsigned C = c * 0x01010101u;
    return f_bits4(f_zero(w.x ^ C)) | (f_bits4(f_zero(w.y ^ C)) << 4) |
           (f_bits4(f_zero(w.z ^ C)) << 8) | (f_bits4(f_zero(w.w ^ C)) << 12);
}
// 0x80 in every byte below 0x21
__device__ __forceinline__ unsigned f_low(unsigned x) {
    return ~((x | 0x80808080u) - 0x21212121u) & ~x & 0x80808080u;
}

__device__ __forceinline__ unsigned f_valid(long long ab, long long n) {
    if (ab + 16 <= n) return 0xFFFFu;
    if (ab >= n) return 0u;
    return (1u << (unsigned)(n - ab)) - 1u;
}

// One vector's masks (byte j in bit j): newlines and dropped separators
// (bytes past the end count as separators); then, given whether byte 0
// starts a line, its line starts and header starts.
struct Vec {
    unsigned nl, sep, ls, H;
};
__device__ __forceinline__ void f_seps(Vec &v, const uint4 &w, unsigned valid) {
    v.nl = 0u;
    v.sep = 0u;
    const unsigned l0 = f_low(w.x), l1 = f_low(w.y), l2 = f_low(w.z), l3 = f_low(w.w);
    if ((l0 | l1 | l2 | l3) != 0u) {
        // the common case: every byte below 0x21 is a newline
        const unsigned N = 0x0A0A0A0Au;
        const unsigned d = (f_zero(w.x ^ N) ^ l0) | (f_zero(w.y ^ N) ^ l1) |
                           (f_zero(w.z ^ N) ^ l2) | (f_zero(w.w ^ N) ^ l3);
        if (d == 0u) {
            const unsigned low = f_bits4(l0) | (f_bits4(l1) << 4) | (f_bits4(l2) << 8) |
                                 (f_bits4(l3) << 12);
            v.nl = low & valid;
            v.sep = low;
        } else {
            v.nl = f_eq16(w, '\n') & valid;
            v.sep = v.nl | f_eq16(w, '\r') | f_eq16(w, ' ') | f_eq16(w, '\t');
        }
    }
    v.sep = (v.sep | ~valid) & 0xFFFFu;
}
// byte j of the vector
__device__ __forceinline__ unsigned f_byte(const uint4 &w, int j) {
    const unsigned wd = (j < 8) ? ((j < 4) ? w.x : w.y) : ((j < 12) ? w.z : w.w);
    return (wd >> (8 * (j & 3))) & 0xFFu;
}
__device__ __forceinline__ void f_lines(Vec &v, const uint4 &w, unsigned valid, unsigned ls0) {
    v.ls = ((v.nl << 1) | ls0) & valid;
    if (v.ls == 0u) v.H = 0u;
    else if ((v.ls & (v.ls - 1u)) == 0u) v.H = (f_byte(w, __ffs(v.ls) - 1) == '>') ? v.ls : 0u;
    else v.H = f_eq16(w, '>') & v.ls;
}
// the kind of the vector's last line start
__device__ __forceinline__ unsigned f_kind(const Vec &v) {
    if (!v.ls) return LS_NONE;
    return ((v.H >> (31 - __clz(v.ls))) & 1u) ? LS_HDR : LS_SEQ;
}
// kept bytes when the vector is entered inside a header (hd) or not: a
// header covers its bytes from its start up to its newline (one subtraction
// per vector: each borrow stops at the newline that ends its line)
__device__ __forceinline__ unsigned f_kept(const Vec &v, bool hd) {
    const unsigned hv = v.H | ((hd && !(v.ls & 1u)) ? 1u : 0u);
    const unsigned E = v.nl | 0x10000u;
    const unsigned cov = (E - hv) & ~E & 0xFFFFu;
    return ~(v.sep | cov) & 0xFFFFu;
}

// The lanes' line starts (any, header) as two ballots; a lane is entered
// inside a header when the last lane below it with a line start has a
// header there, or, with none below it, when the round was.
struct LaneLines {
    unsigned any, hdr;
};
__device__ __forceinline__ LaneLines lane_lines(unsigned kind) {
    return LaneLines{__ballot_sync(kFull, kind != LS_NONE), __ballot_sync(kFull, kind == LS_HDR)};
}
__device__ __forceinline__ bool lane_hd_in(const LaneLines &b, int lane, bool hd_round) {
    const unsigned below = b.any & ((1u << lane) - 1u);
    return below ? ((b.hdr >> (31 - __clz(below))) & 1u) != 0u : hd_round;
}
// the state after the whole round
__device__ __forceinline__ bool round_hd_out(const LaneLines &b, bool hd_round) {
    return b.any ? ((b.hdr >> (31 - __clz(b.any))) & 1u) != 0u : hd_round;
}
// inclusive sum over the warp's lanes
__device__ __forceinline__ unsigned warp_sum_incl(unsigned x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

struct FastaParams {
    const uint8_t *bytes;  // 16-byte aligned
    long long n;
    long long n_spans;
    uint8_t *cbytes;       // kept bytes out
    long long *cso;        // record starts in kept bytes (capacity cso_cap), then the total
    long long cso_cap;
    long long n_ctas;      // CTAs of the sum and emit kernels (8 spans each)
    uint4 *ssum;           // per span: {kept, kept if entered in a header, headers, kind}
    uint4 *csum;           // per CTA: the same over its spans
    longlong2 *sin;        // per CTA: {kept offset, 2 * headers before + in header}
    long long *info;       // the I_* words
    const Carry *cin;      // the scan state before the chunk (stream chunks), or null
    int k;
    int end_boundary;      // the text ends with the chunk (the last record closes)
    unsigned *gate;        // set to `epoch` when the general path must run
    unsigned epoch;
};

// A run of spans as a function of its entry state (inside a header or not).
struct Run2 {
    unsigned kind;              // of the run's last line start (LS_NONE: none)
    long long k_sq, k_hd, heads;  // kept bytes entered outside / inside a header
};
__device__ __forceinline__ Run2 run_identity() { return Run2{LS_NONE, 0, 0, 0}; }
__device__ __forceinline__ Run2 run_of(const uint4 &u) {
    return Run2{u.w, (long long)u.x, (long long)u.y, (long long)u.z};
}
__device__ __forceinline__ bool hd_after(const Run2 &a, bool hd) {
    return a.kind ? a.kind == LS_HDR : hd;
}
// a, then b
__device__ __forceinline__ Run2 run_then(const Run2 &a, const Run2 &b) {
    Run2 r;
    r.kind = b.kind ? b.kind : a.kind;
    r.k_sq = a.k_sq + (hd_after(a, false) ? b.k_hd : b.k_sq);
    r.k_hd = a.k_hd + (hd_after(a, true) ? b.k_hd : b.k_sq);
    r.heads = a.heads + b.heads;
    return r;
}
__device__ __forceinline__ Run2 run_shfl_up(const Run2 &a, int o) {
    Run2 r;
    r.kind = __shfl_up_sync(kFull, a.kind, o);
    r.k_sq = __shfl_up_sync(kFull, a.k_sq, o);
    r.k_hd = __shfl_up_sync(kFull, a.k_hd, o);
    r.heads = __shfl_up_sync(kFull, a.heads, o);
    return r;
}
// the state along the text: inside a header, kept bytes and headers so far
struct TextAt {
    bool hd;
    long long kept, heads;
};
__device__ __forceinline__ TextAt text_then(const TextAt &t, const Run2 &a) {
    return TextAt{hd_after(a, t.hd), t.kept + (t.hd ? a.k_hd : a.k_sq), t.heads + a.heads};
}

// Whether byte s0 starts a line: byte s0 - 1 is '\n', or s0 = 0 and the text
// starts here or the chunk before ended at a line start.
__device__ __forceinline__ unsigned line_start_at(const FastaParams &p, long long s0) {
    if (s0 == 0) return (!p.cin || p.cin->hstate == HS_LS) ? 1u : 0u;
    return p.bytes[s0 - 1] == '\n' ? 1u : 0u;
}

// Per span, entered outside a header: its kept bytes, the kept bytes a span
// entered inside a header drops (those before its first newline, unless its
// byte 0 starts a line), its header starts and the kind of its last line
// start (returned to every lane; lane 0 also stores it).
__device__ __forceinline__ uint4 span_sum(const FastaParams &p, long long span, int lane) {
    const long long s0 = span * kFSpan;
    uint4 w[kFRounds];
#pragma unroll
    for (int r = 0; r < kFRounds; ++r) {  // every load of the span in flight
        const long long ab = s0 + r * 512 + 16 * lane;
        w[r] = make_uint4(0u, 0u, 0u, 0u);
        if (ab < p.n) w[r] = __ldg(reinterpret_cast<const uint4 *>(p.bytes + ab));
    }
    unsigned carry_nl = line_start_at(p, s0);
    bool seen_nl = carry_nl != 0u;  // byte 0 starts a line: nothing depends on the entry
    bool hd = false;
    unsigned kind = LS_NONE, kept = 0u, drop = 0u, heads = 0u;
#pragma unroll
    for (int r = 0; r < kFRounds; ++r) {
        const long long ab = s0 + r * 512 + 16 * lane;
        const unsigned valid = f_valid(ab, p.n);
        Vec v;
        f_seps(v, w[r], valid);
        const unsigned up = __shfl_up_sync(kFull, v.nl >> 15, 1);
        const unsigned ls0 = lane ? up : carry_nl;
        carry_nl = __shfl_sync(kFull, v.nl >> 15, 31);
        f_lines(v, w[r], valid, ls0);
        const LaneLines bl = lane_lines(f_kind(v));
        kept += __popc(f_kept(v, lane_hd_in(bl, lane, hd)));
        heads += __popc(v.H);
        if (!seen_nl) {  // warp-uniform
            const unsigned b = __ballot_sync(kFull, v.nl != 0u);
            const int f = b ? __ffs(b) - 1 : 32;
            const unsigned nonsep = ~v.sep & 0xFFFFu;
            if (lane < f) drop += __popc(nonsep);
            else if (lane == f) drop += __popc(nonsep & ((1u << (__ffs(v.nl) - 1)) - 1u));
            seen_nl = b != 0u;
        }
        if (bl.any) kind = ((bl.hdr >> (31 - __clz(bl.any))) & 1u) ? LS_HDR : LS_SEQ;
        hd = round_hd_out(bl, hd);
    }
    kept = __reduce_add_sync(kFull, kept);
    drop = __reduce_add_sync(kFull, drop);
    heads = __reduce_add_sync(kFull, heads);
    const uint4 u = make_uint4(kept, kept - drop, heads, kind);
    if (lane == 0) p.ssum[span] = u;
    return u;
}

// Every span's summary, and every CTA's (its eight spans in order), the
// scan's input.
__global__ void __launch_bounds__(kFT, 4) fasta_sum_kernel(FastaParams p) {
    __shared__ uint4 s_sum[kFWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long span = (long long)blockIdx.x * kFWarps + warp;
    uint4 u = make_uint4(0u, 0u, 0u, 0u);  // the identity past the end
    if (span < p.n_spans) u = span_sum(p, span, lane);
    if (lane == 0) s_sum[warp] = u;
    __syncthreads();
    if (threadIdx.x == 0) {  // the CTA's spans in order: one summary for the scan
        Run2 t = run_identity();
        for (int w = 0; w < kFWarps; ++w) t = run_then(t, run_of(s_sum[w]));
        p.csum[blockIdx.x] = make_uint4((unsigned)t.k_sq, (unsigned)t.k_hd, (unsigned)t.heads, t.kind);
    }
}

// Symbol code (as the general kernel's carry holds them: 0-3 for A C G T in
// either case, 4 for any other kept byte) and back to a letter.
__device__ __forceinline__ unsigned sym_code(unsigned b) {
    switch (b | 0x20u) {
    case 'a': return 0u;
    case 'c': return 1u;
    case 'g': return 2u;
    case 't': return 3u;
    default: return 4u;
    }
}
__device__ __forceinline__ uint8_t sym_letter(unsigned c) {
    return (c & 4u) ? (uint8_t)'N' : (uint8_t)"ACGT"[c & 3u];
}

__device__ __forceinline__ void decline(const FastaParams &p) {
    p.info[I_N] = 0;
    p.info[I_NREC] = 0;
    *(volatile unsigned *)p.gate = p.epoch;
}

// After the scan (one thread): the chunk's records -- the one continued from
// the chunk before (or an implicit first one when the text starts here and
// byte 0 is not '>'), then one per header -- the symbols of the continued
// record's partial k-mer, written as letters in front of the kept bytes, the
// end of the direct kernels' input (the open last record cut to whole k-mers
// unless the text ends with this chunk; when that record starts at a header
// the emit kernel cuts it), and the line state after the chunk.  The gate is
// raised instead when the direct path cannot take the chunk.
__device__ void scan_totals(const FastaParams &p, const TextAt &at) {
    long long m = 0, d_base = 0, g0 = 0, rec0;
    unsigned long long codes = 0ull;
    if (p.cin) {
        m = p.cin->a.t % p.k;
        d_base = p.cin->a.d;
        g0 = p.cin->a.nb;
        codes = p.cin->a.codes;
        rec0 = 1;
    } else {
        rec0 = (p.bytes[0] != '>') ? 1 : 0;
    }
    const long long n_rec = rec0 + at.heads;
    const long long end = m + at.kept;
    long long n_direct = end;
    if (!p.end_boundary) n_direct = at.heads == 0 ? end / p.k * p.k : -1;
    if (n_rec < 1 || n_rec + 1 > p.cso_cap || n_rec > kMaxRecords || n_direct == 0 ||
        (p.end_boundary && end == 0)) {
        decline(p);
        return;
    }
    p.info[I_NREC] = n_rec;
    p.info[I_START] = kHead - m;
    p.info[I_DBASE] = d_base;
    p.info[I_M] = m;
    p.info[I_G0] = g0;
    p.info[I_CONT] = p.cin ? 1 : 0;
    p.info[I_END] = end;
    p.info[I_HSTATE] = (p.bytes[p.n - 1] == '\n') ? HS_LS : (at.hd ? HS_HD : HS_SQ);
    p.info[I_REC0] = rec0;
    if (rec0) p.cso[0] = 0;
    if (n_direct > 0) {
        p.info[I_N] = n_direct;
        p.cso[n_rec] = n_direct;
    }
    for (long long i = 0; i < m; ++i)  // the carried symbols, oldest first
        p.cbytes[kHead - m + i] = sym_letter((unsigned)(codes >> (3 * (m - 1 - i))) & 7u);
}

// One block: every CTA's incoming (inside a header, kept offset, headers
// before); the totals.  The CTA summaries go through shared memory in tiles
// of kScanTile, loaded and stored coalesced: thread i composes entries
// kScanPer * i .. of the tile, warp scans and then warp 0 over the warps order
// the threads, and the running state carries from tile to tile.
constexpr int kScanPer = 2;
constexpr int kScanTile = kScanT * kScanPer;

__global__ void __launch_bounds__(kScanT) fasta_scan_kernel(FastaParams p) {
    __shared__ uint4 tile_s[kScanTile];  // summaries in, then incoming states out
    __shared__ Run2 wsum[kScanT / 32];
    __shared__ Run2 s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // entered inside a header only when the chunk before ended inside one
    TextAt at{p.cin != nullptr && p.cin->hstate == HS_HD, 0, 0};
    for (long long base = 0; base < p.n_ctas; base += kScanTile) {
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const long long i = base + j * kScanT + tid;
            tile_s[j * kScanT + tid] = (i < p.n_ctas) ? p.csum[i] : make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        uint4 mine[kScanPer];
        Run2 t = run_identity();
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            mine[j] = tile_s[tid * kScanPer + j];
            t = run_then(t, run_of(mine[j]));
        }
        Run2 x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Run2 y = run_shfl_up(x, o);
            if (lane >= o) x = run_then(y, x);
        }
        Run2 ex = run_shfl_up(x, 1);
        if (lane == 0) ex = run_identity();
        if (lane == 31) wsum[warp] = x;
        __syncthreads();  // tile_s reads and wsum writes are done
        if (warp == 0) {
            Run2 z = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const Run2 y = run_shfl_up(z, o);
                if (lane >= o) z = run_then(y, z);
            }
            Run2 zex = run_shfl_up(z, 1);
            if (lane == 0) zex = run_identity();
            if (lane == 31) s_total = z;
            __syncwarp();
            wsum[lane] = zex;  // every warp's exclusive prefix
        }
        __syncthreads();
        TextAt me = text_then(text_then(at, wsum[warp]), ex);
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const longlong2 v = make_longlong2(me.kept, 2 * me.heads + (me.hd ? 1 : 0));
            tile_s[tid * kScanPer + j] = *reinterpret_cast<const uint4 *>(&v);
            me = text_then(me, run_of(mine[j]));
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const long long i = base + j * kScanT + tid;
            if (i < p.n_ctas) p.sin[i] = *reinterpret_cast<const longlong2 *>(&tile_s[j * kScanT + tid]);
        }
        at = text_then(at, s_total);
        __syncthreads();  // tile_s, wsum and s_total are reused by the next tile
    }
    if (tid == 0) scan_totals(p, at);
}

// The 16 bytes of w with the bytes of `keep` packed to the front (the bytes
// after them zero).
__device__ __forceinline__ uint4 f_pack(const uint4 &w, unsigned keep) {
    if (keep == 0xFFFFu) return w;
    const unsigned drop = ~keep & 0xFFFFu;
    if ((drop & (drop - 1u)) == 0u) {
        const unsigned x[4] = {w.x, w.y, w.z, w.w};
        unsigned y[4];
        // one byte dropped at d: the bytes above it move down by one
        const int d = __ffs(drop) - 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const unsigned hi_next = (i < 3) ? x[i + 1] : 0u;
            const unsigned shifted = __funnelshift_r(x[i], hi_next, 8);  // bytes 4i+1 .. 4i+4
            const int lo = d - 4 * i;  // bytes of word i below d stay
            unsigned below;
            if (lo <= 0) below = 0u;
            else if (lo >= 4) below = 0xFFFFFFFFu;
            else below = (1u << (8 * lo)) - 1u;
            y[i] = (x[i] & below) | (shifted & ~below);
        }
        return make_uint4(y[0], y[1], y[2], y[3]);
    }
    // several bytes dropped (header lines, CRLF): byte by byte, in 64-bit
    // halves (no indexed arrays: they would live in local memory)
    const unsigned long long xl = ((unsigned long long)w.y << 32) | w.x;
    const unsigned long long xh = ((unsigned long long)w.w << 32) | w.z;
    unsigned long long yl = 0ull, yh = 0ull;
    int o = 0;
    for (unsigned m = keep; m; m &= m - 1u, ++o) {
        const int j = __ffs(m) - 1;
        const unsigned long long b = ((j < 8) ? (xl >> (8 * j)) : (xh >> (8 * (j - 8)))) & 0xFFull;
        if (o < 8) yl |= b << (8 * o);
        else yh |= b << (8 * (o - 8));
    }
    return make_uint4((unsigned)yl, (unsigned)(yl >> 32), (unsigned)yh, (unsigned)(yh >> 32));
}

// Per span: its vectors' kept bytes at their kept offsets, and its record
// starts.  The warp's window holds the output from the 16-byte boundary at or
// below the round's first kept byte; each lane ORs its packed bytes in at
// their place (up to five words), whole 16-byte pieces go out as vector
// stores, the partial piece at the end moves to the window's front for the
// next round.  The span's first and last pieces may hold bytes of the
// neighbouring spans: only this span's bytes of them are stored, one by one.
__global__ void __launch_bounds__(kFT, 4) fasta_emit_kernel(FastaParams p) {
    __shared__ __align__(16) unsigned win[kFWarps][kWinWords];
    if (*(volatile const unsigned *)p.gate == p.epoch) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long span = (long long)blockIdx.x * kFWarps + warp;
    if (span >= p.n_spans) return;  // warp-level work only: no block barrier below
    const long long s0 = span * kFSpan;
    // three rounds in flight: a ring of registers shifted by one each round
    auto load = [&](int r) {
        const long long ab = s0 + r * 512 + 16 * lane;
        uint4 x = make_uint4(0u, 0u, 0u, 0u);
        if (r < kFRounds && ab < p.n) x = __ldg(reinterpret_cast<const uint4 *>(p.bytes + ab));
        return x;
    };
    uint4 w0 = load(0), w1 = load(1), w2 = load(2);
    unsigned *const wb = win[warp];
    for (int i = lane; i < kWinWords; i += 32) wb[i] = 0u;
    // this span's incoming state: the CTA's, then the CTA's spans before it
    // (lane j holds span j's summary; folded in order)
    const longlong2 in = p.sin[blockIdx.x];
    TextAt at{(in.y & 1) != 0, in.x, in.y >> 1};
    {
        const uint4 mine = (lane < warp) ? p.ssum[(long long)blockIdx.x * kFWarps + lane]
                                         : make_uint4(0u, 0u, 0u, 0u);
        for (int j = 0; j < warp; ++j) {
            uint4 u;
            u.x = __shfl_sync(kFull, mine.x, j);
            u.y = __shfl_sync(kFull, mine.y, j);
            u.z = __shfl_sync(kFull, mine.z, j);
            u.w = __shfl_sync(kFull, mine.w, j);
            at = text_then(at, run_of(u));
        }
    }
    const long long o_begin = at.kept;  // the span's first kept byte
    long long o_cur = at.kept;          // kept offset at the round's start
    bool hd = at.hd;
    long long rec = p.info[I_REC0] + at.heads;
    unsigned carry_nl = line_start_at(p, s0);
    __syncwarp();
#pragma unroll 1
    for (int r = 0; r < kFRounds; ++r) {
        const uint4 wr = w0;
        w0 = w1;
        w1 = w2;
        w2 = load(r + 3);
        const long long ab = s0 + r * 512 + 16 * lane;
        const unsigned valid = f_valid(ab, p.n);
        Vec v;
        f_seps(v, wr, valid);
        const unsigned up = __shfl_up_sync(kFull, v.nl >> 15, 1);
        const unsigned ls0 = lane ? up : carry_nl;
        carry_nl = __shfl_sync(kFull, v.nl >> 15, 31);
        f_lines(v, wr, valid, ls0);
        const LaneLines bl = lane_lines(f_kind(v));
        const unsigned keep = f_kept(v, lane_hd_in(bl, lane, hd));
        const unsigned cnt = __popc(keep);
        const unsigned cinc = warp_sum_incl(cnt, lane);
        const long long o_lane = o_cur + (cinc - cnt);
        const long long o_end = o_cur + __shfl_sync(kFull, cinc, 31);
        if (__ballot_sync(kFull, v.H != 0u)) {
            // record starts: each header's position among the kept bytes
            // (after the carried symbols); the counts are read here, in this
            // rare branch, to keep them out of the loop's registers
            const long long n_rec = p.info[I_NREC], m = p.info[I_M];
            const unsigned nh = __popc(v.H);
            const unsigned hinc = warp_sum_incl(nh, lane);
            long long ri = rec + (hinc - nh);
            for (unsigned hh = v.H; hh; hh &= hh - 1u, ++ri) {
                const int h = __ffs(hh) - 1;
                const long long pos = m + o_lane + __popc(keep & ((1u << h) - 1u));
                if (ri < n_rec) p.cso[ri] = pos;
                if (ri == n_rec - 1 && !p.end_boundary) {
                    // the open last record: its whole k-mers only
                    const long long cut = pos + (p.info[I_END] - pos) / p.k * p.k;
                    if (cut == 0) {
                        *(volatile unsigned *)p.gate = p.epoch;
                    } else {
                        p.info[I_N] = cut;
                        p.cso[n_rec] = cut;
                    }
                }
            }
            rec += __shfl_sync(kFull, hinc, 31);
        }
        const long long wbase = o_cur & ~15ll;  // the window's first byte
        if (cnt) {
            const uint4 pk = f_pack(wr, keep);
            const int off = (int)(o_lane - wbase);
            const int sh = 8 * (off & 3);
            const unsigned q[4] = {pk.x, pk.y, pk.z, pk.w};
            const int first = off >> 2, last = (off + (int)cnt - 1) >> 2;
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const unsigned lo = (i < 4) ? q[i] : 0u;
                const unsigned hi = (i > 0) ? q[i - 1] : 0u;
                const unsigned word = sh ? ((lo << sh) | (hi >> (32 - sh))) : lo;
                if (first + i <= last) atomicOr(&wb[first + i], word);
            }
        }
        __syncwarp();
        const int nfull = (int)((o_end - wbase) >> 4);  // whole pieces in the window
        for (int i = lane; i < nfull; i += 32) {
            const long long ga = wbase + 16 * i;
            const uint4 val = reinterpret_cast<const uint4 *>(wb)[i];
            if (ga >= o_begin) {
                *reinterpret_cast<uint4 *>(p.cbytes + kHead + ga) = val;
            } else {
                const unsigned long long lo = ((unsigned long long)val.y << 32) | val.x;
                const unsigned long long hi = ((unsigned long long)val.w << 32) | val.z;
                for (int j = (int)(o_begin - ga); j < 16; ++j)
                    p.cbytes[kHead + ga + j] = (uint8_t)((j < 8) ? (lo >> (8 * j)) : (hi >> (8 * (j - 8))));
            }
        }
        // the partial piece to the front, the rest cleared
        unsigned keep_w = 0u;
        if (lane < 4) keep_w = wb[4 * nfull + lane];
        __syncwarp();
        for (int i = 4 + lane; i < 4 * nfull + 4; i += 32) wb[i] = 0u;
        if (lane < 4) wb[lane] = keep_w;
        __syncwarp();
        o_cur = o_end;
        hd = round_hd_out(bl, hd);
    }
    // the span's last partial piece
    const long long wbase = o_cur & ~15ll;
    if (lane < 16) {
        const long long ga = wbase + lane;
        if (ga < o_cur && ga >= o_begin)
            p.cbytes[kHead + ga] = (uint8_t)(wb[lane >> 2] >> (8 * (lane & 3)));
    }
}

// Stream chunks, after the direct kernels (one block): each record that
// starts in the chunk gets its first id written at its global boundary index
// (and the end boundary its total when the text ends here); the running
// totals; and the scan state after the chunk in the general kernel's form
// (boundaries, ids, the open record's symbols and their last k - 1 codes,
// the line state), so that either path can take the next chunk.  Nothing
// when the direct path declined the chunk: the general kernel behind writes
// all of it.
__global__ void __launch_bounds__(256) fasta_finish_kernel(FastaParams p, const long long *plan,
                                                           long long *offsets, long long offsets_cap,
                                                           long long *totals, Carry *cout) {
    if (*(volatile const unsigned *)p.gate == p.epoch) return;
    const long long n_rec = p.info[I_NREC], cont = p.info[I_CONT], g0 = p.info[I_G0];
    for (long long r = cont + threadIdx.x; r < n_rec; r += blockDim.x) {
        const long long g = g0 + r - cont;
        if (g < offsets_cap) offsets[g] = plan[r];
    }
    if (threadIdx.x != 0) return;
    const long long d_total = plan[n_rec];
    const long long nb = g0 + (n_rec - cont) + (p.end_boundary ? 1 : 0);
    if (p.end_boundary && nb - 1 < offsets_cap) offsets[nb - 1] = d_total;
    if (totals) {
        totals[0] = d_total;
        totals[1] = nb > 0 ? nb - 1 : 0;
    }
    if (!cout) return;
    const long long end = p.info[I_END], m = p.info[I_M];
    const bool cont_last = cont && n_rec == 1;  // the last record is the continued one
    const long long s_last = p.cso[n_rec - 1];
    Carry c;
    c.a.nb = nb;
    c.a.h = 0;
    c.a.d = d_total;
    c.a.t = cont_last ? p.cin->a.t + (end - m) : end - s_last;
    // the last k - 1 symbols: this chunk's (for the continued record, its
    // new ones only), after the earlier ones when the record continues
    const uint8_t *sym = p.cbytes + kHead - m;
    long long from = cont_last ? m : s_last;
    if (end - from > p.k - 1) from = end - (p.k - 1);
    unsigned long long bits = 0ull;
    for (long long i = from; i < end; ++i) bits = (bits << 3) | sym_code(sym[i]);
    const unsigned long long mine = ((unsigned long long)(end - from) << 58) | bits;
    c.a.codes = cont_last ? codes_concat(p.cin->a.codes, mine, p.k) : mine;
    c.hstate = (unsigned)p.info[I_HSTATE];
    c.pad = 0u;
    *cout = c;
}

}  // namespace

void fasta_destroy(dnatok_handle *h) {
    if (!h->fasta) return;
    cudaFree(h->fasta->cbytes);
    cudaFree(h->fasta->cso);
    cudaFree(h->fasta->ssum);
    cudaFree(h->fasta->csum);
    cudaFree(h->fasta->sin);
    cudaFree(h->fasta->info);
    cudaFree(h->fasta->plan);
    delete h->fasta;
    h->fasta = nullptr;
}

dnatok_status fasta_reserve(dnatok_handle *h, long long n_bytes, long long offsets_cap,
                            cudaStream_t s) {
    if (!h->fasta) {
        h->fasta = new (std::nothrow) FastaState();
        if (!h->fasta) return fail(h, DNATOK_ERR_NOMEM, "host allocation failed");
    }
    FastaState &f = *h->fasta;
    const long long spans = (n_bytes + kFSpan - 1) / kFSpan;
    long long cso_need = offsets_cap < kMaxRecords + 1 ? offsets_cap : kMaxRecords + 1;
    if (cso_need < 1) cso_need = 1;
    const bool grow = n_bytes + 64 > f.cbytes_cap || spans > f.spans_cap ||
                      cso_need > f.cso_cap || !f.info;
    if (!grow) return DNATOK_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(h, DNATOK_ERR_STATE,
                    "workspace must grow during stream capture; call dnatok_reserve first");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaDeviceSynchronize");
    if (n_bytes + 64 > f.cbytes_cap) {
        cudaFree(f.cbytes);
        f.cbytes = nullptr;
        f.cbytes_cap = 0;
        const long long c = n_bytes + n_bytes / 8 + 64;
        e = cudaMalloc(&f.cbytes, (size_t)c);
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMalloc(FASTA kept bytes)");
        f.cbytes_cap = c;
    }
    if (spans > f.spans_cap) {
        cudaFree(f.ssum);
        cudaFree(f.csum);
        cudaFree(f.sin);
        f.ssum = nullptr;
        f.csum = nullptr;
        f.sin = nullptr;
        f.spans_cap = 0;
        const long long c = spans + spans / 8 + 8;
        const long long cc = (c + kFWarps - 1) / kFWarps;
        e = cudaMalloc(&f.ssum, sizeof(uint4) * (size_t)c);
        if (e == cudaSuccess) e = cudaMalloc(&f.csum, sizeof(uint4) * (size_t)cc);
        if (e == cudaSuccess) e = cudaMalloc(&f.sin, sizeof(longlong2) * (size_t)cc);
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMalloc(FASTA span scratch)");
        f.spans_cap = c;
        f.ctas_cap = cc;
    }
    if (cso_need > f.cso_cap) {
        cudaFree(f.cso);
        f.cso = nullptr;
        f.cso_cap = 0;
        e = cudaMalloc(&f.cso, sizeof(long long) * (size_t)cso_need);
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMalloc(FASTA record starts)");
        f.cso_cap = cso_need;
    }
    if (!f.info) {
        e = cudaMalloc(&f.info, kInfo * sizeof(long long));
        if (e == cudaSuccess) e = cudaMalloc(&f.plan, (kMaxRecords + 2) * sizeof(long long));
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMalloc(FASTA counts)");
    }
    return DNATOK_OK;
}

// The compacted path takes one-shot k-mer encodes (k >= 2) of 16-byte
// aligned FASTA text from kFastaMin bytes up to 4 GiB (the per-span counts
// are 32-bit, the kept offsets 64-bit).
bool fasta_direct_eligible(const dnatok_handle *h, int mode, int k, const uint8_t *bytes,
                           long long n) {
    return h->direct && mode == MODE_KMER && k >= 2 && ((uintptr_t)bytes & 15u) == 0 &&
           n >= kFastaMin && n < (1ll << 32) - 1024;
}

// FASTA text -> kept bytes and record starts (three kernels), then the direct
// k-mer kernels over them with their byte and record counts read on the
// device.  A one-shot encode (no carries) has its id offsets and totals
// written by the direct plan; a stream chunk (a carry in, or the stream's
// first chunk with a carry out) continues the open record of the chunk
// before and has them written by the finish kernel, which also writes the
// carry out.  When the direct path cannot take the text (the id offsets'
// capacity, more records than the plan takes, nothing to encode) the scan
// raises the gate instead and every later kernel of the direct path returns
// at once.
dnatok_status fasta_direct(dnatok_handle *h, const uint8_t *bytes, long long n, void *out,
                           long long out_cap, long long *offsets_out, long long offsets_cap,
                           long long *totals_out, const Carry *carry_in, Carry *carry_out,
                           int start_boundary, int end_boundary, unsigned epoch, int k,
                           cudaStream_t s) {
    (void)start_boundary;  // implied: a stream's first chunk has no carry in
    const bool stream = carry_in || carry_out;
    dnatok_status st = fasta_reserve(h, n, stream ? kMaxRecords + 1 : offsets_cap, s);
    if (st != DNATOK_OK) return st;
    FastaState &f = *h->fasta;
    FastaParams p;
    p.bytes = bytes;
    p.n = n;
    p.n_spans = (n + kFSpan - 1) / kFSpan;
    p.cbytes = f.cbytes;
    p.cso = f.cso;
    p.cso_cap = (stream || offsets_cap > f.cso_cap) ? f.cso_cap : offsets_cap;
    p.n_ctas = (p.n_spans + kFWarps - 1) / kFWarps;
    p.ssum = f.ssum;
    p.csum = f.csum;
    p.sin = f.sin;
    p.info = f.info;
    p.cin = carry_in;
    p.k = k;
    p.end_boundary = end_boundary;
    p.gate = h->d_gate;
    p.epoch = epoch;
    const unsigned grid = (unsigned)p.n_ctas;
    fasta_sum_kernel<<<grid, kFT, 0, s>>>(p);
    fasta_scan_kernel<<<1, kScanT, 0, s>>>(p);
    fasta_emit_kernel<<<grid, kFT, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e, "FASTA compaction launch");
    // the kept bytes begin kHead - I_M bytes into the buffer: n + 32 bytes
    // and kMaxRecords records bound the device-side counts
    e = launch_direct(MODE_KMER, f.cbytes, n + 2 * kHead, f.cso, kMaxRecords, out,
                      stream ? f.plan : offsets_out, stream ? nullptr : totals_out, h->d_gate,
                      epoch, k, h->d_lut, h->sm_count, h->dshape, s, f.info, out_cap);
    if (e != cudaSuccess) return fail_cuda(h, e, "direct kernel launch");
    if (stream) {
        fasta_finish_kernel<<<1, 256, 0, s>>>(p, f.plan, offsets_out, offsets_cap, totals_out,
                                              carry_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail_cuda(h, e, "FASTA finish launch");
    }
    return DNATOK_OK;
}

}  // namespace dnatok
