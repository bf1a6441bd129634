// tile_kernel.cuh -- the single-launch byte -> token-ID kernel.
//
// One persistent grid walks chunks (NSUB consecutive byte-balanced tiles) of
// the flat byte stream in increasing order: chunks are claimed from an atomic
// counter, so every chunk a CTA waits on is held by a running CTA, and
// several CTAs share each SM so one CTA's waits overlap another's work.
// Tiles reach shared memory by 1-D TMA bulk copies (plain loads fetch the
// ragged head and tail), double-buffered so the next tile's copy overlaps the
// current tile's work.  Per chunk:
//   0. FASTA only: each 16-byte vector's line-state map is composed in byte
//      order (warp shuffles, then across warps), the chunk's map is published
//      and a look-back over the predecessors' maps gives the line state at
//      the chunk start;
//   1. pass 1 reads the chunk's tiles from HBM and computes only the chunk's
//      scan element (records, kept symbols, completed tokens, trailing
//      partial k-mer): for RAW input a vector without a byte below 0x21 is
//      kept whole, so this pass is a cheap separator test plus the record
//      boundaries (found by a 32-way search of seq_offsets);
//   2. the chunk's scan element is published and one warp runs a decoupled
//      look-back, 128 predecessors per round trip (self-validating tagged
//      descriptors), while the copy of the chunk's first tile is in flight
//      again;
//   3. pass 2 re-reads the tiles (from L2: this SM read them moments ago),
//      classifies each 16-byte vector four bytes per 32-bit operation -- the
//      2-bit codes are ((b >> 1) ^ (b >> 2)) & 3, and the canonical letter
//      rebuilt from the codes by a byte permute marks, exactly, which bytes
//      are A/C/G/T in either case (the rest form an N bit plane); only vectors
//      holding separators or header bytes take a per-byte path through the
//      256-entry class table -- packs the kept symbols as 2-bit codes by
//      tile-kept index (a warp/block scan of kept counts and a shifted OR when
//      something is dropped), and emits the tokens with the prefix carried
//      from tile to tile: one thread per 16-symbol word, every k-mer whose
//      LAST kept symbol lies in the word being a 2k-bit field of one 64-bit
//      window of the packed codes (leading symbols from before the tile come
//      from the prefix's partial k-mer); record tails (UNK) and id offsets
//      are written per boundary.
// Ownership by last symbol means no tile reads past its own end, and the
// carry between chunks of a stream is just the last chunk's inclusive prefix.
//
// Paper: the device-side ascii_lut[Bytes] gather of the bytes path (Sec. 2.2,
// Algorithm 2) and MapKmer (Algorithm 2) on ragged and FASTA input; the
// k-mer id is the closed form sum_i 4^(k-1-i) * code(b_i).
#pragma once
#include "common.cuh"

namespace dnatok {

enum : int { BSRC_LIST = 0, BSRC_FASTA = 1, BSRC_FLAGS = 2 };

struct TileParams {
    const uint8_t *bytes;          // chunk bytes (device)
    long long n_bytes;             // chunk length
    const long long *seq_offsets;  // BSRC_LIST: n_bnd sorted boundary positions
    long long n_bnd;
    void *out;                     // int32 ids, or uint8 symbols (MODE_SYM)
    long long out_cap;
    long long *offsets_out;        // boundary index -> token index
    long long offsets_cap;
    long long *totals_out;         // {tokens, records} or null
    TileDesc *desc;
    unsigned long long *tile_counter;  // [0] claim counter, [1] exit counter
    const Carry *carry_in;         // null = start of a stream
    Carry *carry_out;              // null = not needed
    int *status;
    const int *lut;                // MODE_CHAR: 256 ids on the device
    long long n_tiles;
    long long n_chunks;            // chunks of NSUB tiles (the unit of the look-back)
    unsigned epoch;
    int k;
    int start_boundary;            // boundary at the chunk's first byte (non-list sources)
    int end_boundary;              // boundary after the chunk's last byte (non-list sources)
    int head_pad;                  // (uintptr_t)bytes & 15
    int lut_keeps_bases;           // MODE_CHAR: the table keeps all of A C G T a c g t
    const unsigned *gate;          // non-null: run only if *gate == gate_epoch
    unsigned gate_epoch;
    long long spin_limit;          // polls before a look-back wait gives up (DEV_TIMEOUT)
    long long skip_chunk;          // >= 0: this chunk is left unprocessed (wait-limit tests)
    unsigned *clear_gate;          // non-null (captured launches behind the direct path):
                                   // after a run, the last CTA clears *clear_gate and the
                                   // chunk descriptors, so the next replay starts clean
};

constexpr int kMaxB = 256;     // segments per emission round
constexpr int kChunkB = 1024;  // record boundaries of a chunk kept in shared memory

// Shared memory (dynamic) of one CTA.
__host__ __device__ constexpr int tile_smem_bytes(int tile, int nt) {
    return 2 * tile                      // two TMA buffers
           + 4 * (tile / 16 + 2)         // packed codes P (one leading word)
           + 2 * (tile / 16 + 4)         // N bit plane, 16 bits per word
           + 8 * (tile / 16)             // kmask, kpre, bmask, bpre (u16)
           + 4 * kChunkB                 // the chunk's record boundaries
           + 13 * (kMaxB + 1)            // segment table
           + 256;
}

// -------------------------------------------------------------- SWAR helpers

// 2-bit codes of four bytes (A/a 0, C/c 1, G/g 2, T/t 3), one per byte lane.
__device__ __forceinline__ unsigned codes4(unsigned x) {
    return ((x >> 1) ^ (x >> 2)) & 0x03030303u;
}
// 0x80 in every byte lane that is NOT one of A/C/G/T/a/c/g/t: the uppercase
// letter of each lane's code is rebuilt with a byte permute of "ACGT" and
// compared with the byte folded to upper case.
__device__ __forceinline__ unsigned nonbase4(unsigned x, unsigned c) {
    const unsigned t = c | (c >> 4);                    // nibbles c0 c1 . c2 c3 ...
    const unsigned sel = __byte_perm(t, 0, 0x0020);     // nibbles c0 c1 c2 c3
    const unsigned u = __byte_perm(0x54474341u, 0, sel);
    const unsigned d = (x & 0xDFDFDFDFu) ^ u;
    return (((d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | d) & 0x80808080u;
}
// 0x80 in every byte lane whose value is below 0x21 (space and controls).
__device__ __forceinline__ unsigned low4(unsigned x) {
    return ~((x | 0x80808080u) - 0x21212121u) & ~x & 0x80808080u;
}
// 0x80 in every byte lane of t that is zero.
__device__ __forceinline__ unsigned zero4(unsigned t) {
    return ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u;
}
// 0x80 in every byte lane that is one of the four separators (C3).
__device__ __forceinline__ unsigned sep4(unsigned x) {
    if (!low4(x)) return 0u;
    return zero4(x ^ 0x09090909u) | zero4(x ^ 0x0A0A0A0Au) | zero4(x ^ 0x0D0D0D0Du) |
           zero4(x ^ 0x20202020u);
}
// High bits of the four byte lanes -> 4 bits, byte 0 in bit 0.
__device__ __forceinline__ unsigned gather4(unsigned m) {
    return (((m >> 7) & 0x01010101u) * 0x01020408u) >> 24;
}
// Separator lanes of a 16-byte vector as 16 bits (byte j in bit j).
__device__ __forceinline__ unsigned sepmask16(const uint4 &w) {
    return gather4(sep4(w.x)) | (gather4(sep4(w.y)) << 4) | (gather4(sep4(w.z)) << 8) |
           (gather4(sep4(w.w)) << 12);
}
__device__ __forceinline__ bool has_byte16(const uint4 &w, unsigned pat) {
    return (zero4(w.x ^ pat) | zero4(w.y ^ pat) | zero4(w.z ^ pat) | zero4(w.w ^ pat)) != 0u;
}
// Remove the symbols whose bits are set in `drop` (16-bit, symbol j in bit j)
// from 16 MSB-first 2-bit codes and from an LSB-first 16-bit flag word.
__device__ __forceinline__ void compact16(unsigned drop, unsigned &codes, unsigned &flags) {
    while (drop) {
        const int j = 31 - __clz(drop);  // highest first: lower indices stay put
        drop &= ~(1u << j);
        const unsigned hi = j ? (0xFFFFFFFFu << (32 - 2 * j)) : 0u;
        codes = (codes & hi) | ((codes << 2) & ~hi);
        const unsigned lo = (1u << j) - 1u;
        flags = (flags & lo) | ((flags >> 1) & ~lo);
    }
}
// Four byte-lane codes -> one byte, first byte in the two top bits.
__device__ __forceinline__ unsigned pack4(unsigned c) {
    const unsigned r = __byte_perm(c, 0, 0x0123);
    const unsigned m = r | (r >> 6);
    return (m & 0xFu) | ((m >> 12) & 0xF0u);
}

// -------------------------------------------------------------- warp scans

__device__ __forceinline__ unsigned warp_incl_scan(unsigned x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned warp_incl_hmap(unsigned m) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, m, o);
        if (lane >= o) m = hmap_compose(y, m);
    }
    return m;
}

// Ordered exclusive scan of one value per vector, vectors ordered
// (warp, iteration, lane).  s_w needs NW + 1 slots.  Returns the total.
template <int NT, int VPT>
__device__ __forceinline__ unsigned block_scan_vec(const unsigned (&v)[VPT], unsigned (&ex)[VPT],
                                                   unsigned *s_w) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned run = 0;
#pragma unroll
    for (int it = 0; it < VPT; ++it) {
        unsigned inc = warp_incl_scan(v[it]);
        ex[it] = run + inc - v[it];
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncthreads();
    if (lane == 0) s_w[warp] = run;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < NW ? s_w[lane] : 0u;
        unsigned inc = warp_incl_scan(w);
        if (lane < NW) s_w[lane] = inc - w;
        if (lane == 31) s_w[NW] = inc;
    }
    __syncthreads();
    unsigned off = s_w[warp];
#pragma unroll
    for (int it = 0; it < VPT; ++it) ex[it] += off;
    return s_w[NW];
}

// Same for line-state maps (composition, applied in byte order).
template <int NT, int VPT>
__device__ __forceinline__ unsigned block_scan_hmap(const unsigned (&v)[VPT], unsigned (&ex)[VPT],
                                                    unsigned *s_w) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned run = kHmapIdentity;
#pragma unroll
    for (int it = 0; it < VPT; ++it) {
        unsigned inc = warp_incl_hmap(v[it]);
        unsigned before = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) before = kHmapIdentity;
        ex[it] = hmap_compose(run, before);
        run = hmap_compose(run, __shfl_sync(0xffffffffu, inc, 31));
    }
    __syncthreads();
    if (lane == 0) s_w[warp] = run;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < NW ? s_w[lane] : kHmapIdentity;
        unsigned inc = warp_incl_hmap(w);
        unsigned before = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) before = kHmapIdentity;
        if (lane < NW) s_w[lane] = before;
        if (lane == 31) s_w[NW] = inc;
    }
    __syncthreads();
    unsigned off = s_w[warp];
#pragma unroll
    for (int it = 0; it < VPT; ++it) ex[it] = hmap_compose(off, ex[it]);
    return s_w[NW];
}

// First index i in [0, n) with off[i] >= x (n if none); one full warp, a
// 32-way search (three rounds of loads for a few thousand entries).
__device__ __forceinline__ long long warp_lower_bound(const long long *off, long long n,
                                                      long long x) {
    const int lane = threadIdx.x & 31;
    long long lo = 0, hi = n;  // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const long long step = (hi - lo + 31) >> 5;
        const long long idx = lo + lane * step;
        const bool less = idx < hi && off[idx] < x;
        const int c = __popc(__ballot_sync(0xffffffffu, less));
        const long long nlo = c ? lo + (long long)(c - 1) * step + 1 : lo;
        long long nhi = lo + (long long)c * step;
        if (nhi > hi) nhi = hi;
        lo = nlo;
        hi = nhi;
    }
    const long long idx = lo + lane;
    const bool less = idx < hi && off[idx] < x;
    return lo + __popc(__ballot_sync(0xffffffffu, less));
}

// --------------------------------------------------------------- look-back

// Decoupled look-back over the tagged count descriptors (one full warp; each
// lane reads four consecutive predecessors, so one round trip covers 128).
// Only the tiles after the nearest inclusive prefix must have published.
// Returns the exclusive prefix of tile t; on a timeout records DEV_TIMEOUT
// and returns the identity.
static __device__ __noinline__ Agg lookback_counts(const TileParams &p, long long t,
                                                    const Agg &carry) {
    const int lane = threadIdx.x & 31;
    const int k = p.k;
    const KDiv kd = make_kdiv(k);
    Agg acc = agg_identity();
    long long base = t;
    for (;;) {
        const long long idx0 = base - 128 + 4 * lane;
        const unsigned ep = p.epoch & ((1u << kEpochBits) - 1);
        Agg mine;
        int spins = 0, sleep_ns = 32;
        int lstar;
        for (;;) {
            // cheap poll: the tag word of each of this lane's four tiles
            unsigned fl[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long idx = idx0 + j;
                if (idx >= 0) {
                    const unsigned tg = (unsigned)(ld_relaxed_u64(p.desc[idx].w) >> 44);
                    fl[j] = ((tg >> 2) == ep) ? (tg & 3u) : LB_EMPTY;
                    if (fl[j] != LB_AGG && fl[j] != LB_INCL) fl[j] = LB_EMPTY;
                } else {
                    fl[j] = LB_INCL;  // before the chunk: the carry, then nothing
                }
            }
            int hi = -1;
            bool empty_above = false;
#pragma unroll
            for (int j = 3; j >= 0; --j) {
                if (hi >= 0) continue;
                if (fl[j] == LB_INCL) hi = j;
                else if (fl[j] == LB_EMPTY) empty_above = true;
            }
            const unsigned has_incl = __ballot_sync(0xffffffffu, hi >= 0);
            lstar = has_incl ? 31 - __clz(has_incl) : -1;
            // only the tiles after the nearest inclusive prefix must be ready
            bool ok = lane < lstar || !empty_above;
            if (__all_sync(0xffffffffu, ok)) {
                // full read of the tiles this lane contributes, folded backward
                mine = agg_identity();
                if (lane >= lstar) {
#pragma unroll
                    for (int j = 3; j >= 0; --j) {
                        if (j < (hi < 0 ? 0 : hi)) continue;
                        const long long idx = idx0 + j;
                        Agg a;
                        if (idx >= 0) {
                            unsigned long long w0, w1, w2, w3;
                            ld_relaxed_v2u64(p.desc[idx].w, w0, w1);
                            ld_relaxed_v2u64(p.desc[idx].w + 2, w2, w3);
                            // a torn or changed slot sends the whole warp back to polling
                            if (decode_desc(w0, w1, w2, w3, p.epoch, k, a) != fl[j]) ok = false;
                        } else {
                            a = (idx == -1) ? carry : agg_identity();
                        }
                        mine = agg_combine(a, mine, kd);
                    }
                }
                if (__all_sync(0xffffffffu, ok)) break;
            }
            if (++spins > p.spin_limit || dev_failed(p.status)) {
                if (lane == 0) set_dev_status(p.status, DEV_TIMEOUT);
                return agg_identity();
            }
            __nanosleep(sleep_ns);
            if (sleep_ns < 1024) sleep_ns <<= 1;
        }
        if (lane < lstar) mine = agg_identity();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Agg u = shfl_up_agg(mine, o);
            if (lane >= o) mine = agg_combine(u, mine, kd);
        }
        const Agg win = shfl_agg(mine, 31);
        acc = agg_combine(win, acc, kd);
        if (lstar >= 0) return acc;
        base -= 128;
    }
}

// Look-back over the FASTA line-state maps.  Returns the line state at the
// start of tile t.
static __device__ unsigned lookback_hmap(const TileParams &p, long long t, unsigned carry_state) {
    const int lane = threadIdx.x & 31;
    const unsigned ep = p.epoch & 0xffffffu;
    unsigned acc = kHmapIdentity;
    long long base = t;
    for (;;) {
        const long long idx = base - 32 + lane;
        unsigned flag = LB_INCL, m = kHmapIdentity;
        if (idx == -1) m = hmap_const(carry_state);
        int spins = 0;
        unsigned incl;
        int jstar;
        for (;;) {
            if (idx >= 0) {
                unsigned hs = ld_acquire_u32(&p.desc[idx].hstatus);
                flag = ((hs >> 8) == ep) ? ((hs >> 6) & 3u) : LB_EMPTY;
                m = hs & 63u;
            }
            incl = __ballot_sync(0xffffffffu, flag == LB_INCL);
            const unsigned empty = __ballot_sync(0xffffffffu, flag == LB_EMPTY);
            jstar = incl ? 31 - __clz(incl) : -1;
            const unsigned above = (jstar >= 31) ? 0u : (0xffffffffu << (jstar + 1));
            if (!(empty & above)) break;
            if (++spins > p.spin_limit || dev_failed(p.status)) {
                if (lane == 0) set_dev_status(p.status, DEV_TIMEOUT);
                return HS_LS;
            }
            __nanosleep(spins < 32 ? 32 : 256);
        }
        if (lane < jstar) m = kHmapIdentity;
        m = warp_incl_hmap(m);
        unsigned win = __shfl_sync(0xffffffffu, m, 31);
        acc = hmap_compose(win, acc);
        if (incl) return hmap_apply(acc, HS_LS);
        base -= 32;
    }
}

// -------------------------------------------------------------- the kernel

template <int MODE, int BSRC, int NT, int TILE, int NSUB>
__global__ void __launch_bounds__(NT, 1024 / NT) tile_kernel(const TileParams p) {
    constexpr int NV = TILE / 16;
    constexpr int VPT = NV / NT;
    constexpr int NW = NT / 32;
    static_assert(VPT >= 1 && NV % NT == 0 && NW >= 4, "tile / thread shape");
    constexpr bool PACKED = (MODE == MODE_KMER || MODE == MODE_SYM);
    // behind the direct path: run only when it found its premise broken
    if (p.gate) {
        pdl_wait();
        if (*(volatile const unsigned *)p.gate != p.gate_epoch) return;
    }

    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *tbuf0 = smem;
    unsigned *Pw = reinterpret_cast<unsigned *>(smem + 2 * TILE);  // NV + 2 words
    unsigned *P = Pw + 1;                                          // P[-1] is the prefix
    uint16_t *NBw = reinterpret_cast<uint16_t *>(Pw + NV + 2);     // NV + 4 halves
    uint16_t *NB16 = NBw + 2;  // 4-byte aligned (also read as 32-bit words); NB16[-1] is the prefix
    uint16_t *kmask = NBw + NV + 4;
    uint16_t *kpre = kmask + NV;
    uint16_t *bmask = kpre + NV;
    uint16_t *bpre = bmask + NV;
    unsigned *cbpos = reinterpret_cast<unsigned *>(bpre + NV);        // [kChunkB]
    unsigned *sks = cbpos + kChunkB;                                  // segment start
    unsigned *sL = sks + (kMaxB + 1);                                 // segment length
    unsigned *sC = sL + (kMaxB + 1);                                  // token base in tile
    uint8_t *sJr = reinterpret_cast<uint8_t *>(sC + (kMaxB + 1));     // phase at start

    __shared__ uint64_t mbar[2];
    __shared__ uint8_t cls_s[256];
    __shared__ int lut_s[256];
    __shared__ unsigned s_w[NW + 1];
    __shared__ long long s_chunk, s_crb[2];
    __shared__ long long s_trb[NSUB + 1];
    __shared__ Agg s_tagg[NSUB];
    __shared__ Agg s_prefix, s_cagg;
    __shared__ long long s_T0, s_R0, s_ttok;
    __shared__ unsigned long long s_pcodes;
    __shared__ unsigned s_Jr;
    __shared__ unsigned s_tmap[NSUB + 1], s_hchunk, s_hend;
    __shared__ long long s_red[NW];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = (MODE == MODE_KMER) ? p.k : 1;
    const KDiv kd = make_kdiv(k);
    const unsigned kmagic = kd.m32;  // n / k = umulhi(n, kmagic) for n < 2^17, k >= 2

    for (int i = tid; i < 256; i += NT) {
        uint8_t c;
        switch (i) {
        case 'A': case 'a': c = 0; break;
        case 'C': case 'c': c = 1; break;
        case 'G': case 'g': c = 2; break;
        case 'T': case 't': c = 3; break;
        case '\n': c = CB_SEP | CB_NL; break;
        case '\r': case ' ': case '\t': c = CB_SEP; break;
        case '>': c = CB_N | CB_GT; break;
        default: c = CB_N;
        }
        cls_s[i] = c;
        if (MODE == MODE_CHAR) lut_s[i] = p.lut[i];
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }

    const uint8_t *abase = p.bytes - p.head_pad;
    const long long end_rel = (long long)p.head_pad + p.n_bytes;
    const Agg carry = p.carry_in ? p.carry_in->a : agg_identity();
    const unsigned carry_h = p.carry_in ? p.carry_in->hstate : HS_LS;
    unsigned phase[2] = {0u, 0u};
    int buf = 0;
    bool in_flight[2] = {false, false};

    auto tile_vlo = [&](long long t) -> int {
        const long long rel_lo = t * TILE;
        return (int)((rel_lo < p.head_pad ? p.head_pad : rel_lo) - rel_lo);
    };
    auto tile_vhi = [&](long long t) -> int {
        const long long rel_lo = t * TILE;
        return (int)((rel_lo + TILE < end_rel ? rel_lo + TILE : end_rel) - rel_lo);
    };
    // Issue the copy of tile t into buffer b (thread 0), plus plain loads of
    // its ragged ends (threads 0..31).
    auto stage = [&](long long t, int b) {
        const long long rel_lo = t * TILE;
        const int vlo = tile_vlo(t), vhi = tile_vhi(t);
        const int a_lo = (vlo + 15) & ~15, a_hi = vhi & ~15;
        uint8_t *tb = tbuf0 + b * TILE;
        if (tid == 0) {
            bulk_wait_read();  // a bulk store from this buffer must have read it
            // the ragged ends (first and last tile of the input only)
            for (int i = vlo; i < (a_lo < vhi ? a_lo : vhi); ++i) tb[i] = abase[rel_lo + i];
            for (int i = (a_lo > a_hi ? a_lo : a_hi); i < vhi; ++i)
                if (i >= vlo) tb[i] = abase[rel_lo + i];
            fence_proxy_async_shared();
            if (a_hi > a_lo) {
                mbar_arrive_expect_tx(&mbar[b], (unsigned)(a_hi - a_lo));
                tma_load_1d(tb + a_lo, abase + rel_lo + a_lo, (unsigned)(a_hi - a_lo), &mbar[b]);
            } else {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&mbar[b]))
                             : "memory");
            }
        }
        in_flight[b] = true;
    };
    auto wait_buf = [&](int b) {
        int spins = 0;
        while (!mbar_try_wait(&mbar[b], phase[b])) {
            if (++spins > kSpinLimit) {  // a bulk copy that never lands: give up
                set_dev_status(p.status, DEV_TIMEOUT);
                break;
            }
        }
        phase[b] ^= 1u;
        in_flight[b] = false;
    };

    __syncthreads();
    bool failed = dev_failed(p.status);

    while (!failed) {
        if (tid == 0) s_chunk = (long long)atomicAdd(&p.tile_counter[0], 1ull);
        __syncthreads();
        const long long c = s_chunk;
        if (c >= p.n_chunks) break;
        if (c == p.skip_chunk) {  // never published: the next chunk's look-back runs out
            __syncthreads();
            continue;
        }
        const long long t0 = c * NSUB;
        const int nt = (int)((p.n_tiles - t0) < NSUB ? (p.n_tiles - t0) : NSUB);
        const long long cbyte0 = t0 * TILE - p.head_pad;  // chunk index of tile t0's byte 0
        const int n_items = (BSRC == BSRC_FASTA ? nt : 0) + 2 * nt;
        auto item_tile = [&](int it) -> long long {
            return t0 + ((BSRC == BSRC_FASTA) ? it % nt : (it < nt ? it : it - nt));
        };
        stage(item_tile(0), buf);

        // ------------------------------------------- record boundaries (RAW)
        if (BSRC == BSRC_LIST) {
            if (warp == 1) {
                const long long first = cbyte0 < 0 ? 0 : cbyte0;
                const long long r = warp_lower_bound(p.seq_offsets, p.n_bnd, first);
                if (lane == 0) s_crb[0] = r;
            } else if (warp == 2) {
                long long r = p.n_bnd;
                if (t0 + nt < p.n_tiles)
                    r = warp_lower_bound(p.seq_offsets, p.n_bnd, cbyte0 + (long long)nt * TILE);
                if (lane == 0) s_crb[1] = r;
            }
            __syncthreads();
            const long long lo = s_crb[0], hi = s_crb[1];
            long long first = cbyte0 < 0 ? 0 : cbyte0;
            long long last = cbyte0 + (long long)nt * TILE;
            if (last > p.n_bytes) last = p.n_bytes;
            bool bad = hi < lo;
            for (long long i = tid; lo + i < hi; i += NT) {
                const long long a = p.seq_offsets[lo + i];
                if (a < first || a > last) bad = true;
                if (lo + i > 0 && p.seq_offsets[lo + i - 1] > a) bad = true;
                if (lo + i == 0 && a != 0) bad = true;
                if (lo + i == p.n_bnd - 1 && a != p.n_bytes) bad = true;
                if (i < kChunkB) {
                    long long pos = a - cbyte0;  // relative to tile t0's byte 0
                    pos = pos < 0 ? 0 : (pos > (long long)nt * TILE ? (long long)nt * TILE : pos);
                    cbpos[i] = (unsigned)pos;
                }
            }
            if (bad) set_dev_status(p.status, DEV_BAD_OFFSETS);
            __syncthreads();
            // each tile's first boundary: lower bound of its first byte
            if (tid <= nt) {
                const int i = tid;
                long long r;
                if (i == nt) {
                    r = hi;
                } else if (i == 0) {
                    r = lo;
                } else {
                    const long long x = (long long)i * TILE;  // relative to tile t0's byte 0
                    long long a = 0, b = hi - lo;
                    while (a < b) {
                        const long long m = (a + b) >> 1;
                        const long long v = (m < kChunkB) ? (long long)cbpos[m]
                                                          : p.seq_offsets[lo + m] - cbyte0;
                        if (v < x) a = m + 1; else b = m;
                    }
                    r = lo + a;
                }
                s_trb[i] = r;
            }
        }

        Agg cagg = agg_identity();
        unsigned hrun = kHmapIdentity;
        for (int it = 0; it < n_items; ++it) {
            const int pass = (BSRC == BSRC_FASTA) ? (it / nt) : (it < nt ? 1 : 2);
            const int ti = (BSRC == BSRC_FASTA) ? it % nt : (it < nt ? it : it - nt);
            const long long t = t0 + ti;
            const int vlo = tile_vlo(t), vhi = tile_vhi(t);
            const int cur = buf;
            const uint8_t *tb = tbuf0 + cur * TILE;
            wait_buf(cur);
            __syncthreads();
            buf ^= 1;  // the next item goes to the other buffer
            if (it + 1 < n_items) stage(item_tile(it + 1), buf);

            // ------------------------------------------------ FASTA line states
            unsigned hin[VPT];
            if (BSRC == BSRC_FASTA) {
                unsigned m[VPT];
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    const int v = warp * 32 * VPT + q * 32 + lane;
                    unsigned s0 = HS_LS, s1 = HS_HD, s2 = HS_SQ;
                    const uint4 w4 = *reinterpret_cast<const uint4 *>(tb + 16 * v);
                    const bool full = (16 * v >= vlo) && (16 * v + 16 <= vhi);
                    // Only '\n' and '>' move the line state.  Without a '>',
                    // a vector with no newline maps LS -> SQ (its first byte
                    // starts a sequence line) and keeps HD and SQ; with one, the
                    // state after its last newline is LS if that newline is the
                    // vector's last byte, else SQ.
                    if (full && !has_byte16(w4, 0x3E3E3E3Eu)) {
                        if (!has_byte16(w4, 0x0A0A0A0Au)) {
                            m[q] = HS_SQ | (HS_HD << 2) | (HS_SQ << 4);
                        } else {
                            const unsigned e = (w4.w >> 24) == 0x0Au ? HS_LS : HS_SQ;
                            m[q] = e | (e << 2) | (e << 4);
                        }
                    } else {
                        for (int j = 0; j < 16; ++j) {
                            const int i = 16 * v + j;
                            if (i >= vlo && i < vhi) {
                                const uint8_t b = tb[i];
                                s0 = hstep(s0, b); s1 = hstep(s1, b); s2 = hstep(s2, b);
                            }
                        }
                        m[q] = s0 | (s1 << 2) | (s2 << 4);
                    }
                }
                const unsigned tmap = block_scan_hmap<NT, VPT>(m, hin, s_w);
                if (pass == 0) {
                    if (tid == 0) {
                        s_tmap[ti] = hrun;
                        hrun = hmap_compose(hrun, tmap);
                        s_tmap[ti + 1] = hrun;
                    }
                    if (ti == nt - 1) {
                        // the chunk's line state: publish its map, look back
                        __syncthreads();
                        if (warp == 0) {
                            const unsigned cmap = s_tmap[nt];
                            unsigned x;
                            if (c == 0) {
                                x = carry_h;
                            } else {
                                if (lane == 0)
                                    st_release_u32(&p.desc[c].hstatus,
                                                   ((p.epoch & 0xffffffu) << 8) | (LB_AGG << 6) | cmap);
                                x = lookback_hmap(p, c, carry_h);
                            }
                            if (lane == 0) {
                                const unsigned xe = hmap_apply(cmap, x);
                                st_release_u32(&p.desc[c].hstatus, ((p.epoch & 0xffffffu) << 8) |
                                                                       (LB_INCL << 6) | hmap_const(xe));
                                s_hchunk = x;
                                s_hend = xe;
                            }
                        }
                    }
                    __syncthreads();
                    continue;
                }
                const unsigned x_t = hmap_apply(s_tmap[ti], s_hchunk);
#pragma unroll
                for (int q = 0; q < VPT; ++q) hin[q] = hmap_apply(hin[q], x_t);
            }

            // -------------------------------------------------- classify (SWAR)
            const bool full_pass = (pass == 2);
            unsigned pc[VPT], nb16[VPT], sepm[VPT];
            bool slow[VPT], med[VPT];
            bool tile_plain = (vlo == 0 && vhi == TILE);
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                const int v = warp * 32 * VPT + q * 32 + lane;
                const uint4 w4 = *reinterpret_cast<const uint4 *>(tb + 16 * v);
                const bool full = (16 * v >= vlo) && (16 * v + 16 <= vhi);
                bool s = !full;
                bool md = false;
                pc[q] = 0u;
                nb16[q] = 0u;
                sepm[q] = 0u;
                if (MODE == MODE_CHAR && !p.lut_keeps_bases) {
                    s = true;
                } else if (BSRC == BSRC_FASTA && PACKED && !full_pass) {
                    // pass 1 of FASTA input needs kept counts only: outside
                    // header lines every byte but a separator is kept (the
                    // scan element's trailing codes are read from the bytes)
                    const unsigned sm = sepmask16(w4);
                    const bool gt = has_byte16(w4, 0x3E3E3E3Eu);
                    if (sm || gt) {
                        s = true;
                        if (full && !gt && hin[q] != HS_HD) {
                            md = true;
                            sepm[q] = sm;
                        }
                    }
                } else if (full_pass || BSRC == BSRC_FASTA || MODE == MODE_CHAR) {
                    const unsigned c0 = codes4(w4.x), c1 = codes4(w4.y);
                    const unsigned c2 = codes4(w4.z), c3 = codes4(w4.w);
                    const unsigned n0 = nonbase4(w4.x, c0), n1 = nonbase4(w4.y, c1);
                    const unsigned n2 = nonbase4(w4.z, c2), n3 = nonbase4(w4.w, c3);
                    if (PACKED)
                        pc[q] = (pack4(c0) << 24) | (pack4(c1) << 16) | (pack4(c2) << 8) | pack4(c3);
                    if (n0 | n1 | n2 | n3) {
                        nb16[q] = gather4(n0) | (gather4(n1) << 4) | (gather4(n2) << 8) |
                                  (gather4(n3) << 12);
                        if (BSRC == BSRC_FASTA || MODE == MODE_CHAR) {
                            s = true;  // header bytes / table ids depend on the byte itself
                        } else if ((low4(w4.x) & n0) | (low4(w4.y) & n1) | (low4(w4.z) & n2) |
                                   (low4(w4.w) & n3)) {
                            s = true;  // a separator (or a control byte) is present
                        }
                        // separators and N-class bytes only, and no header can
                        // start or continue here: the SWAR compaction path
                        if (PACKED && s && full &&
                            (BSRC != BSRC_FASTA ||
                             (hin[q] != HS_HD && !has_byte16(w4, 0x3E3E3E3Eu)))) {
                            md = true;
                            sepm[q] = sepmask16(w4);
                        }
                    }
                } else {
                    // pass 1 of RAW input: only separators change the kept counts
                    if (low4(w4.x) | low4(w4.y) | low4(w4.z) | low4(w4.w)) {
                        s = true;
                        if (PACKED && full) {
                            md = true;
                            sepm[q] = sepmask16(w4);
                        }
                    }
                }
                if (BSRC == BSRC_FASTA && hin[q] == HS_HD) s = true;  // inside a header line
                if (BSRC != BSRC_LIST && p.start_boundary && t == 0 && 16 * v <= vlo &&
                    vlo < 16 * v + 16) {
                    s = true;
                    md = false;
                }
                slow[q] = s;
                med[q] = md && s;
                tile_plain &= !s;
            }
            if (BSRC == BSRC_FASTA) tile_plain = false;

            // ---------------------------------------- kept symbols and placement
            const bool fast = __syncthreads_and(tile_plain) != 0;
            unsigned K = (unsigned)(vhi - vlo);
            unsigned NBb = 0;
            if (fast) {
                if (PACKED && full_pass) {
#pragma unroll
                    for (int q = 0; q < VPT; ++q) {
                        const int v = warp * 32 * VPT + q * 32 + lane;
                        P[v] = pc[q];
                        NB16[v] = (uint16_t)nb16[q];
                    }
                }
            } else {
                unsigned km[VPT], bm[VPT], kc[VPT], kx[VPT], bc[VPT], bx[VPT];
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    const int v = warp * 32 * VPT + q * 32 + lane;
                    if (!slow[q]) {
                        km[q] = 0xFFFFu;
                        bm[q] = 0u;
                    } else if (med[q]) {
                        km[q] = ~sepm[q] & 0xFFFFu;
                        bm[q] = 0u;
                        if (PACKED && full_pass) {
                            unsigned cw = pc[q], nf = nb16[q] & ~sepm[q];
                            compact16(sepm[q], cw, nf);
                            pc[q] = cw;
                            nb16[q] = nf;
                        }
                    } else {
                        unsigned kmv = 0, bmv = 0, acc = 0, nac = 0, n = 0;
                        unsigned s = (BSRC == BSRC_FASTA) ? hin[q] : 0u;
                        for (int j = 0; j < 16; ++j) {
                            const int i = 16 * v + j;
                            if (i < vlo || i >= vhi) continue;
                            const uint8_t b = tb[i];
                            bool hdr = false, bnd = false;
                            if (BSRC == BSRC_FASTA) {
                                bnd = (s == HS_LS && b == '>');
                                hdr = bnd || s == HS_HD;
                                s = hstep(s, b);
                            }
                            if (BSRC != BSRC_LIST && p.start_boundary && t == 0 && i == vlo)
                                bnd = true;
                            const uint8_t cl = cls_s[b];
                            bool kept;
                            if (MODE == MODE_CHAR) kept = !hdr && lut_s[b] >= 0;
                            else kept = !hdr && !(cl & CB_SEP);
                            if (kept) {
                                kmv |= 1u << j;
                                acc = (acc << 2) | (cl & 3u);
                                nac |= (unsigned)((cl >> 2) & 1u) << n;
                                ++n;
                            }
                            bmv |= (unsigned)bnd << j;
                        }
                        km[q] = kmv;
                        bm[q] = bmv;
                        pc[q] = n ? acc << (32 - 2 * n) : 0u;
                        nb16[q] = nac;
                    }
                    kc[q] = __popc(km[q]);
                    bc[q] = __popc(bm[q]);
                }
                K = block_scan_vec<NT, VPT>(kc, kx, s_w);
                if (BSRC != BSRC_LIST) NBb = block_scan_vec<NT, VPT>(bc, bx, s_w);
                if (PACKED && full_pass) {
                    for (int i = tid; i < NV + 1; i += NT) P[i] = 0u;
                    for (int i = tid; i < NV + 2; i += NT) NB16[i] = 0;
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    const int v = warp * 32 * VPT + q * 32 + lane;
                    kmask[v] = (uint16_t)km[q];
                    kpre[v] = (uint16_t)kx[q];
                    if (BSRC != BSRC_LIST) {
                        bmask[v] = (uint16_t)bm[q];
                        bpre[v] = (uint16_t)bx[q];
                    }
                    if (PACKED && full_pass && kc[q]) {
                        const unsigned x = kx[q];
                        const unsigned s = 2 * (x & 15u);
                        atomicOr(&P[x >> 4], pc[q] >> s);
                        if (s) atomicOr(&P[(x >> 4) + 1], pc[q] << (32 - s));
                        if (nb16[q]) {
                            unsigned *NB32 = reinterpret_cast<unsigned *>(NB16);
                            const unsigned sn = x & 31u;
                            atomicOr(&NB32[x >> 5], nb16[q] << sn);
                            if (sn + kc[q] > 32) atomicOr(&NB32[(x >> 5) + 1], nb16[q] >> (32 - sn));
                        }
                    }
                }
            }
            __syncthreads();

            // kept symbols of the tile before tile-local byte index i (vlo <= i <= vhi)
            auto kept_before = [&](int i) -> unsigned {
                if (i >= vhi) return K;
                if (fast) return (unsigned)(i - vlo);
                const int v = i >> 4;
                return (unsigned)kpre[v] + __popc((unsigned)kmask[v] & ((1u << (i & 15)) - 1u));
            };
            auto code_at = [&](int x) -> unsigned { return (P[x >> 4] >> (30 - 2 * (x & 15))) & 3u; };
            auto nflag_at = [&](int x) -> unsigned { return (NB16[x >> 4] >> (x & 15)) & 1u; };

            // boundaries of the tile
            long long rb_lo = 0, nb;
            if (BSRC == BSRC_LIST) {
                rb_lo = s_trb[ti];
                nb = s_trb[ti + 1] - rb_lo;
                if (nb < 0) {
                    set_dev_status(p.status, DEV_BAD_OFFSETS);
                    nb = 0;
                }
            } else {
                nb = (long long)NBb + ((p.end_boundary && t == p.n_tiles - 1) ? 1 : 0);
            }
            const long long crb_lo = (BSRC == BSRC_LIST) ? s_crb[0] : 0;
            auto bnd_pos = [&](long long i) -> int {
                long long pos;
                if (BSRC == BSRC_LIST) {
                    const long long j = rb_lo + i - crb_lo;  // index in the chunk's list
                    pos = ((j < kChunkB) ? (long long)cbpos[j] : p.seq_offsets[rb_lo + i] - cbyte0) -
                          (long long)ti * TILE;
                } else {
                    if (i >= NBb) return vhi;
                    int lo = 0, hi = NV - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (bpre[mid] <= i) lo = mid; else hi = mid - 1;
                    }
                    unsigned m = bmask[lo];
                    for (unsigned r = (unsigned)(i - bpre[lo]); r > 0; --r) m &= m - 1;
                    pos = 16 * lo + __ffs(m) - 1;
                }
                return (int)(pos < vlo ? vlo : (pos > vhi ? vhi : pos));
            };
            auto bnd_kept = [&](long long i) -> unsigned { return kept_before(bnd_pos(i)); };

            if (pass == 1) {
                // ------------------------------------------ the tile's scan element
                long long dsum = 0;
                for (long long i = tid; i + 1 < nb; i += NT) {
                    const unsigned a = bnd_kept(i), b = bnd_kept(i + 1);
                    dsum += b > a ? kd.div32(b - a + k - 1) : 0;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
                if (lane == 0) s_red[warp] = dsum;
                __syncthreads();
                if (tid == 0) {
                    long long d = 0;
                    for (int w = 0; w < NW; ++w) d += s_red[w];
                    Agg a;
                    a.nb = nb;
                    long long open;
                    if (nb == 0) {
                        a.h = K; a.d = 0; a.t = 0; open = K;
                    } else {
                        a.h = bnd_kept(0);
                        a.t = K - bnd_kept(nb - 1);
                        a.d = d + kd.div32((unsigned)a.t);
                        open = a.t;
                    }
                    unsigned long long codes = 0;
                    if (MODE == MODE_KMER && k > 1) {
                        // the last kept symbols, read back from the tile bytes
                        const int n = (int)(open < k - 1 ? open : k - 1);
                        unsigned long long bits = 0;
                        int q = 0;
                        for (int i = vhi - 1; i >= vlo && q < n; --i) {
                            bool kept;
                            if (fast) kept = true;
                            else kept = (kmask[i >> 4] >> (i & 15)) & 1u;
                            if (!kept) continue;
                            const uint8_t cl = cls_s[tb[i]];
                            bits |= (unsigned long long)(cl & 7u) << (3 * q);
                            ++q;
                        }
                        codes = ((unsigned long long)n << 58) | bits;
                    }
                    a.codes = codes;
                    s_tagg[ti] = a;
                    cagg = agg_combine(cagg, a, kd);
                    if (ti == nt - 1) {
                        s_cagg = cagg;
                        if (c > 0) publish_desc(&p.desc[c], cagg, p.epoch, LB_AGG);
                    }
                }
                __syncthreads();
                if (ti == nt - 1) {
                    // ------------------------------------- look back, once per chunk
                    if (warp == 0) {
                        const Agg pre = (c == 0) ? carry : lookback_counts(p, c, carry);
                        if (lane == 0) {
                            const Agg incl = agg_combine(pre, s_cagg, kd);
                            publish_desc(&p.desc[c], incl, p.epoch, LB_INCL);
                            s_prefix = pre;
                            if (c == p.n_chunks - 1) {
                                if (p.totals_out) {
                                    p.totals_out[0] = incl.d;
                                    p.totals_out[1] = incl.nb > 0 ? incl.nb - 1 : 0;
                                }
                                if (p.carry_out) {
                                    Carry cr;
                                    cr.a = incl;
                                    cr.hstate = (BSRC == BSRC_FASTA) ? s_hend : HS_LS;
                                    cr.pad = 0;
                                    *p.carry_out = cr;
                                }
                            }
                        }
                    }
                    __syncthreads();
                    if (dev_failed(p.status)) {
                        failed = true;
                        break;
                    }
                }
                continue;
            }

            // ----------------------------------------------------- emit (pass 2)
            // thread 0 advances the running prefix; everyone reads its fields
            if (tid == 0) {
                const Agg Pf = s_prefix;
                const long long J = (Pf.nb > 0) ? Pf.t : Pf.h;
                const Agg after = agg_combine(Pf, s_tagg[ti], kd);
                s_T0 = (Pf.nb > 0) ? Pf.d : 0;
                s_R0 = Pf.nb;
                s_Jr = (unsigned)(J - kd.div(J) * k);
                s_pcodes = Pf.codes;
                s_ttok = after.d - s_T0;
                s_prefix = after;  // read by no one until the next tile's emission
            }
            __syncthreads();
            const long long T0 = s_T0;
            const long long R0 = s_R0;
            const unsigned Jr = s_Jr;
            if (MODE != MODE_KMER || k == 1) {
                if (MODE == MODE_CHAR && !fast) {
#pragma unroll
                    for (int q = 0; q < VPT; ++q) {
                        const int v = warp * 32 * VPT + q * 32 + lane;
                        unsigned m = kmask[v];
                        long long o = T0 + kpre[v];
                        while (m) {
                            const int j = __ffs(m) - 1;
                            m &= m - 1;
                            if (o < p.out_cap) static_cast<int *>(p.out)[o] = lut_s[tb[16 * v + j]];
                            ++o;
                        }
                    }
                } else {
                    for (unsigned x = tid; x < K; x += NT) {
                        const long long o = T0 + x;
                        if (o >= p.out_cap) break;
                        if (MODE == MODE_CHAR) {
                            static_cast<int *>(p.out)[o] = lut_s[tb[vlo + x]];
                        } else {
                            const unsigned s = nflag_at((int)x) ? 4u : code_at((int)x);
                            if (MODE == MODE_SYM) static_cast<uint8_t *>(p.out)[o] = (uint8_t)s;
                            else static_cast<int *>(p.out)[o] = (int)s;
                        }
                    }
                }
                for (long long i = tid; i < nb; i += NT) {
                    const long long g = R0 + i;
                    if (g < p.offsets_cap) p.offsets_out[g] = T0 + bnd_kept(i);
                }
            } else {
                const unsigned unk = 1u << (2 * k);
                const unsigned cmask = unk - 1u;
                const unsigned nkm = (1u << k) - 1u;
                // The tile's ids are staged in its (now free) byte buffer and leave
                // with one bulk copy when they fit and the output is 16-byte aligned.
                const long long tile_tokens = s_ttok;
                const bool staged = ((reinterpret_cast<uintptr_t>(p.out) & 15u) == 0) &&
                                    tile_tokens + 4 <= TILE / 4;
                int *stg = reinterpret_cast<int *>(tbuf0 + cur * TILE);
                const unsigned shift = (unsigned)(T0 & 3);
                auto put = [&](unsigned u, unsigned id) {  // u: token index within the tile
                    if (staged) {
                        stg[u + shift] = (int)id;
                    } else {
                        const long long o = T0 + u;
                        if (o < p.out_cap) static_cast<int *>(p.out)[o] = (int)id;
                    }
                };
                if (tid == 0) {  // the prefix's partial k-mer becomes word -1
                    const unsigned long long pcodes = s_pcodes;
                    const int cnt = codes_count(pcodes);
                    unsigned w = 0, nbits = 0;
                    for (int q = 0; q < cnt; ++q) {
                        const unsigned s = (unsigned)(pcodes >> (3 * q)) & 7u;
                        w |= (s & 3u) << (2 * q);
                        nbits |= ((s >> 2) & 1u) << (15 - q);
                    }
                    P[-1] = w;
                    NB16[-1] = (uint16_t)nbits;
                }
                unsigned tok_base = 0;
                for (long long seg0 = 0; seg0 < nb + 1; seg0 += kMaxB) {
                    const int nseg = (int)((nb + 1 - seg0) < kMaxB ? (nb + 1 - seg0) : kMaxB);
                    unsigned cnt[1];
                    for (int s = tid; s < nseg; s += NT) {
                        const long long gs = seg0 + s;
                        const unsigned ks = (gs == 0) ? 0u : bnd_kept(gs - 1);
                        const unsigned ke0 = (gs == nb) ? K : bnd_kept(gs);
                        const unsigned ke = ke0 < ks ? ks : ke0;  // only malformed offsets decrease
                        const unsigned jr = (gs == 0) ? Jr : 0u;
                        const unsigned L = ke - ks;
                        const unsigned n = jr + L;
                        const unsigned full = __umulhi(n, kmagic);
                        const unsigned tail = (gs < nb && n != full * k) ? 1u : 0u;
                        sks[s] = ks;
                        sL[s] = L;
                        sJr[s] = (uint8_t)jr;
                        sC[s] = full + tail;
                    }
                    __syncthreads();
                    if (nseg == 1) {
                        cnt[0] = sC[0];
                        __syncthreads();
                        if (tid == 0) sC[0] = 0;
                    } else {
                        unsigned run = 0;
                        for (int b0 = 0; b0 < nseg; b0 += NT) {
                            const int s = b0 + tid;
                            unsigned vv1[1] = {(s < nseg) ? sC[s] : 0u}, ex1[1];
                            const unsigned tot = block_scan_vec<NT, 1>(vv1, ex1, s_w);
                            if (s < nseg) sC[s] = run + ex1[0];
                            run += tot;
                        }
                        cnt[0] = run;
                    }
                    __syncthreads();
                    for (int s = tid; s < nseg; s += NT) {
                        const long long gs = seg0 + s;
                        const unsigned base = tok_base + sC[s];
                        if (gs >= 1 && R0 + gs - 1 < p.offsets_cap)
                            p.offsets_out[R0 + gs - 1] = T0 + base;
                        if (gs < nb) {
                            const unsigned n = sJr[s] + sL[s];
                            const unsigned full = __umulhi(n, kmagic);
                            if (n != full * k) put(base + full, unk);  // the record's tail
                        }
                    }
                    const unsigned kfirst = sks[0];
                    const unsigned klast = sks[nseg - 1] + sL[nseg - 1];
                    if (klast > kfirst) {
                        const unsigned w_lo = kfirst >> 4, w_hi = (klast - 1) >> 4;
                        for (unsigned w = w_lo + tid; w <= w_hi; w += NT) {
                            const unsigned x_lo = 16 * w, x_hi = x_lo + 16;
                            const unsigned whi = P[(int)w - 1], wlo = P[w];
                            const unsigned nwin =
                                (unsigned)NB16[(int)w - 1] | ((unsigned)NB16[w] << 16);
                            int s = 0;
                            if (nseg > 1) {
                                int lo = 0, hi = nseg - 1;
                                while (lo < hi) {
                                    const int mid = (lo + hi + 1) >> 1;
                                    if (sks[mid] <= x_lo) lo = mid; else hi = mid - 1;
                                }
                                s = lo;
                            }
                            for (; s < nseg && sks[s] < x_hi; ++s) {
                                const unsigned ks = sks[s];
                                const unsigned a = ks > x_lo ? ks : x_lo;
                                const unsigned e_end = ks + sL[s];
                                const unsigned b = e_end < x_hi ? e_end : x_hi;
                                if (a >= b) continue;
                                const unsigned n = a - ks + sJr[s];
                                const unsigned q = __umulhi(n, kmagic);
                                const unsigned r = n - q * k;
                                unsigned u = tok_base + sC[s] + q;
                                for (unsigned e = a - x_lo + (k - 1 - r); e < b - x_lo; e += k, ++u) {
                                    // the k-mer ending at symbol x_lo + e: 2k bits of (whi:wlo)
                                    unsigned id = __funnelshift_r(wlo, whi, 30 - 2 * e) & cmask;
                                    if ((nwin >> (17 + e - k)) & nkm) id = unk;
                                    put(u, id);
                                }
                            }
                        }
                    }
                    tok_base += cnt[0];
                    __syncthreads();
                }
                if (staged && tile_tokens > 0) {
                    long long g_lo = T0, g_hi = T0 + tile_tokens;
                    if (g_hi > p.out_cap) g_hi = p.out_cap;
                    const long long a_lo = (g_lo + 3) & ~3ll, a_hi = g_hi & ~3ll;
                    if (tid == 0 && a_hi > a_lo) {
                        fence_proxy_async_shared();
                        tma_store_1d(static_cast<int *>(p.out) + a_lo, stg + (a_lo - T0 + shift),
                                     (unsigned)(4 * (a_hi - a_lo)));
                        bulk_commit();
                    }
                    const long long h_end = a_lo < g_hi ? a_lo : g_hi;
                    const long long t_beg = a_hi > a_lo ? a_hi : a_lo;
                    if (tid >= 32 && tid < 36) {
                        const long long o = g_lo + (tid - 32);
                        if (o < h_end) static_cast<int *>(p.out)[o] = stg[o - T0 + shift];
                    } else if (tid >= 36 && tid < 40) {
                        const long long o = t_beg + (tid - 36);
                        if (o >= g_lo && o < g_hi) static_cast<int *>(p.out)[o] = stg[o - T0 + shift];
                    }
                }
            }
            __syncthreads();
        }
    }

    // Leave no copy in flight: a CTA that stopped early waits (bounded) for it.
    __syncthreads();
    for (int b = 0; b < 2; ++b) {
        if (in_flight[b]) {
            int spins = 0;
            while (!mbar_try_wait(&mbar[b], phase[b]) && ++spins < kSpinLimit) {
            }
        }
    }
    // The last CTA out resets the chunk counters for the next launch.
    __shared__ int s_last;
    __syncthreads();
    if (tid == 0) {
        bulk_wait_all();
        __threadfence();
        const unsigned long long done = atomicAdd(&p.tile_counter[1], 1ull);
        s_last = done == gridDim.x - 1;
        if (s_last) {
            p.tile_counter[0] = 0ull;
            p.tile_counter[1] = 0ull;
            __threadfence();
        }
    }
    if (p.clear_gate) {
        __syncthreads();
        if (s_last) {
            __threadfence();
            uint4 *d = reinterpret_cast<uint4 *>(p.desc);
            const long long nw = p.n_chunks * (long long)(sizeof(TileDesc) / sizeof(uint4));
            for (long long i = tid; i < nw; i += NT) d[i] = make_uint4(0u, 0u, 0u, 0u);
            if (tid == 0) *(volatile unsigned *)p.clear_gate = 0u;
        }
    }
}

}  // namespace dnatok
