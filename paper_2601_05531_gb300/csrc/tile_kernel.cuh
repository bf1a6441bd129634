// tile_kernel.cuh -- the single-pass byte -> token-ID kernel.
//
// One persistent grid walks byte-balanced tiles of the flat byte stream in
// increasing order (tiles are claimed from an atomic counter, so every tile a
// CTA waits on is held by a running CTA).  Per tile:
//   1. a 1-D TMA bulk copy stages the tile's 16-byte-aligned interior into
//      shared memory (plain loads fetch the ragged head and tail);
//   2. FASTA only: each 16-byte vector's line-state map is composed in order
//      (warp shuffles, then across warps) and a first look-back over the
//      predecessors' maps gives the line state at the tile start;
//   3. each byte is classified through a 256-entry table in shared memory
//      (bases, N-class, separators, header bytes, record boundaries); kept
//      bytes are counted and compacted with warp/block scans;
//   4. the tile's scan element (records, kept symbols, completed tokens,
//      trailing partial k-mer) is published and a decoupled look-back over
//      the predecessors' descriptors yields the exclusive prefix;
//   5. every token whose LAST kept symbol lies in the tile is emitted (its
//      leading symbols may come from the prefix's partial k-mer), and every
//      record boundary in the tile writes its id offset.
// Ownership by last symbol means no tile reads past its own end, and the
// carry between chunks of a stream is just the last tile's inclusive prefix.
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
    const int *tile_rec;           // BSRC_LIST: first boundary index per tile (n_tiles + 1)
    void *out;                     // int32 ids, or uint8 symbols (MODE_SYM)
    long long out_cap;
    long long *offsets_out;        // boundary index -> token index
    long long offsets_cap;
    long long *totals_out;         // {tokens, records} or null
    TileDesc *desc;
    unsigned long long *tile_counter;
    const Carry *carry_in;         // null = start of a stream
    Carry *carry_out;              // null = not needed
    int *status;
    const int *lut;                // MODE_CHAR: 256 ids on the device
    long long n_tiles;
    unsigned epoch;
    int k;
    int start_boundary;            // boundary at the chunk's first byte (non-list sources)
    int end_boundary;              // boundary after the chunk's last byte (non-list sources)
    int head_pad;                  // (uintptr_t)bytes & 15
};

__host__ __device__ constexpr int tile_smem_bytes(int tile, int nt) {
    // tb[tile] + cc[tile] + 4 u16 tables of tile/16 + 3 u32 segment arrays
    return 2 * tile + 4 * 2 * (tile / 16) + 3 * 4 * 1024 + 128;
}

constexpr int kSegChunk = 1024;

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

// --------------------------------------------------------------- look-back

// Decoupled look-back over the count descriptors (called by one full warp).
// Returns the exclusive prefix of tile t; on a timeout records DEV_TIMEOUT
// and returns the identity.
static __device__ Agg lookback_counts(const TileParams &p, long long t, const Agg &carry) {
    const int lane = threadIdx.x & 31;
    const unsigned ep = p.epoch & 0x3fffffffu;
    Agg acc = agg_identity();
    long long base = t;
    for (;;) {
        const long long idx = base - 32 + lane;
        unsigned flag = LB_INCL;
        int spins = 0;
        for (;;) {
            if (idx >= 0) {
                unsigned st = ld_acquire_u32(&p.desc[idx].status);
                flag = ((st >> 2) == ep) ? (st & 3u) : LB_EMPTY;
            }
            if (__all_sync(0xffffffffu, flag != LB_EMPTY)) break;
            if (++spins > kSpinLimit || dev_failed(p.status)) {
                if (lane == 0) set_dev_status(p.status, DEV_TIMEOUT);
                return agg_identity();
            }
            __nanosleep(spins < 64 ? 20 : 200);
        }
        Agg v = agg_identity();
        if (idx >= 0)
            v = load_agg(flag == LB_INCL ? &p.desc[idx].incl : &p.desc[idx].agg);
        else if (idx == -1)
            v = carry;
        const unsigned incl = __ballot_sync(0xffffffffu, flag == LB_INCL);
        const int jstar = incl ? 31 - __clz(incl) : -1;
        if (lane < jstar) v = agg_identity();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Agg u = shfl_up_agg(v, o);
            if (lane >= o) v = agg_combine(u, v, p.k);
        }
        Agg win = shfl_agg(v, 31);
        acc = agg_combine(win, acc, p.k);
        if (incl) return acc;
        base -= 32;
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
        for (;;) {
            if (idx >= 0) {
                unsigned hs = ld_acquire_u32(&p.desc[idx].hstatus);
                flag = ((hs >> 8) == ep) ? ((hs >> 6) & 3u) : LB_EMPTY;
                m = hs & 63u;
            }
            if (__all_sync(0xffffffffu, flag != LB_EMPTY)) break;
            if (++spins > kSpinLimit || dev_failed(p.status)) {
                if (lane == 0) set_dev_status(p.status, DEV_TIMEOUT);
                return HS_LS;
            }
            __nanosleep(spins < 64 ? 20 : 200);
        }
        const unsigned incl = __ballot_sync(0xffffffffu, flag == LB_INCL);
        const int jstar = incl ? 31 - __clz(incl) : -1;
        if (lane < jstar) m = kHmapIdentity;
        m = warp_incl_hmap(m);
        unsigned win = __shfl_sync(0xffffffffu, m, 31);
        acc = hmap_compose(win, acc);
        if (incl) return hmap_apply(acc, HS_LS);
        base -= 32;
    }
}

// -------------------------------------------------------------- the kernel

template <int MODE>
__device__ __forceinline__ uint8_t symbol_of(uint8_t b, const uint8_t *cls) {
    if (MODE == MODE_CHAR) return b;                       // raw byte; table applied at emission
    if (MODE == MODE_SYM) return (cls[b] & CB_N) ? 4 : (cls[b] & 3);
    return cls[b] & 7;                                     // KMER: code | N flag
}

template <int MODE, int BSRC, int NT, int TILE>
__global__ void __launch_bounds__(NT) tile_kernel(const TileParams p) {
    constexpr int NV = TILE / 16;
    constexpr int VPT = NV / NT;
    constexpr int NW = NT / 32;
    static_assert(VPT >= 1 && NV % NT == 0, "tile / thread shape");

    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *tb = smem;                                       // tile bytes (TMA target)
    uint8_t *cc = smem + TILE;                                // compacted symbols
    uint16_t *kmask = reinterpret_cast<uint16_t *>(smem + 2 * TILE);
    uint16_t *kpre = kmask + NV;
    uint16_t *bmask = kpre + NV;
    uint16_t *bpre = bmask + NV;
    unsigned *seg_k = reinterpret_cast<unsigned *>(bpre + NV);  // segment start (tile-kept)
    unsigned *seg_l = seg_k + kSegChunk;                        // segment length
    unsigned *seg_c = seg_l + kSegChunk;                        // token count, then exclusive prefix

    __shared__ uint64_t mbar;
    __shared__ uint8_t cls_s[256];
    __shared__ int lut_s[256];
    __shared__ unsigned s_w[NW + 1];
    __shared__ long long s_tile;
    __shared__ Agg s_prefix, s_agg;
    __shared__ unsigned s_hin, s_hend;
    __shared__ long long s_red[NW];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = (MODE == MODE_KMER) ? p.k : 1;

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
        mbar_init(&mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    if (dev_failed(p.status)) return;
    const uint8_t *abase = p.bytes - p.head_pad;
    const Agg carry = p.carry_in ? p.carry_in->a : agg_identity();
    const unsigned carry_h = p.carry_in ? p.carry_in->hstate : HS_LS;
    unsigned phase = 0;

    for (;;) {
        if (tid == 0) s_tile = (long long)atomicAdd(p.tile_counter, 1ull);
        __syncthreads();
        const long long t = s_tile;
        if (t >= p.n_tiles) break;

        // ------------------------------------------------ 1. stage the tile
        const long long rel_lo = t * TILE;
        const long long end_rel = (long long)p.head_pad + p.n_bytes;
        const int vlo = (int)((rel_lo < p.head_pad ? p.head_pad : rel_lo) - rel_lo);
        const int vhi = (int)((rel_lo + TILE < end_rel ? rel_lo + TILE : end_rel) - rel_lo);
        const int a_lo = (vlo + 15) & ~15, a_hi = vhi & ~15;
        if (tid == 0) {
            fence_proxy_async_shared();
            if (a_hi > a_lo) {
                mbar_arrive_expect_tx(&mbar, (unsigned)(a_hi - a_lo));
                tma_load_1d(tb + a_lo, abase + rel_lo + a_lo, (unsigned)(a_hi - a_lo), &mbar);
            } else {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&mbar))
                             : "memory");
            }
        }
        if (tid < 16) {
            int i = vlo + tid;
            if (i < (a_lo < vhi ? a_lo : vhi)) tb[i] = abase[rel_lo + i];
        } else if (tid < 32) {
            int i = (a_lo > a_hi ? a_lo : a_hi) + (tid - 16);
            if (i >= vlo && i < vhi) tb[i] = abase[rel_lo + i];
        }
        {
            int spins = 0;
            while (!mbar_try_wait(&mbar, phase)) {
                if (++spins > kSpinLimit) {  // a bulk copy that never lands: give up
                    set_dev_status(p.status, DEV_TIMEOUT);
                    break;
                }
            }
        }
        phase ^= 1u;
        __syncthreads();

        // ---------------------------------- 2. FASTA line states (look-back #1)
        unsigned hin[VPT];
        if (BSRC == BSRC_FASTA) {
            unsigned m[VPT];
#pragma unroll
            for (int it = 0; it < VPT; ++it) {
                const int v = warp * 32 * VPT + it * 32 + lane;
                unsigned s0 = HS_LS, s1 = HS_HD, s2 = HS_SQ;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int i = 16 * v + j;
                    if (i >= vlo && i < vhi) {
                        const uint8_t b = tb[i];
                        s0 = hstep(s0, b); s1 = hstep(s1, b); s2 = hstep(s2, b);
                    }
                }
                m[it] = s0 | (s1 << 2) | (s2 << 4);
            }
            const unsigned tmap = block_scan_hmap<NT, VPT>(m, hin, s_w);
            if (warp == 0) {
                unsigned x;
                if (t == 0) {
                    x = carry_h;
                } else {
                    if (lane == 0)
                        st_release_u32(&p.desc[t].hstatus,
                                       ((p.epoch & 0xffffffu) << 8) | (LB_AGG << 6) | tmap);
                    x = lookback_hmap(p, t, carry_h);
                }
                if (lane == 0) {
                    const unsigned xe = hmap_apply(tmap, x);
                    st_release_u32(&p.desc[t].hstatus,
                                   ((p.epoch & 0xffffffu) << 8) | (LB_INCL << 6) | hmap_const(xe));
                    s_hin = x;
                    s_hend = xe;
                }
            }
            __syncthreads();
#pragma unroll
            for (int it = 0; it < VPT; ++it) hin[it] = hmap_apply(hin[it], s_hin);
        }

        // --------------------------------------------- 3. classify and count
        unsigned kc[VPT], kx[VPT], bc[VPT], bx[VPT];
        bool all_kept = true;
#pragma unroll
        for (int it = 0; it < VPT; ++it) {
            const int v = warp * 32 * VPT + it * 32 + lane;
            unsigned km = 0, bm = 0, valid = 0;
            unsigned s = (BSRC == BSRC_FASTA) ? hin[it] : 0u;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int i = 16 * v + j;
                if (i < vlo || i >= vhi) continue;
                valid |= 1u << j;
                const uint8_t b = tb[i];
                bool hdr = false, bnd = false;
                if (BSRC == BSRC_FASTA) {
                    bnd = (s == HS_LS && b == '>');
                    hdr = bnd || s == HS_HD;
                    s = hstep(s, b);
                }
                if (BSRC != BSRC_LIST && p.start_boundary && t == 0 && i == vlo) bnd = true;
                bool kept;
                if (MODE == MODE_CHAR) kept = !hdr && lut_s[b] >= 0;
                else kept = !hdr && !(cls_s[b] & CB_SEP);
                km |= (unsigned)kept << j;
                bm |= (unsigned)bnd << j;
            }
            kmask[v] = (uint16_t)km;
            bmask[v] = (uint16_t)bm;
            kc[it] = __popc(km);
            bc[it] = __popc(bm);
            all_kept &= (km == valid);
        }
        const unsigned K = block_scan_vec<NT, VPT>(kc, kx, s_w);
#pragma unroll
        for (int it = 0; it < VPT; ++it) kpre[warp * 32 * VPT + it * 32 + lane] = (uint16_t)kx[it];
        unsigned NBb = 0;
        if (BSRC != BSRC_LIST) {
            NBb = block_scan_vec<NT, VPT>(bc, bx, s_w);
#pragma unroll
            for (int it = 0; it < VPT; ++it)
                bpre[warp * 32 * VPT + it * 32 + lane] = (uint16_t)bx[it];
        }
        all_kept = __syncthreads_and(all_kept);

        // compaction of kept symbols (skipped when every byte is kept)
        if (!all_kept) {
#pragma unroll
            for (int it = 0; it < VPT; ++it) {
                const int v = warp * 32 * VPT + it * 32 + lane;
                unsigned km = kmask[v];
                unsigned o = kx[it];
                while (km) {
                    const int j = __ffs(km) - 1;
                    km &= km - 1;
                    cc[o++] = symbol_of<MODE>(tb[16 * v + j], cls_s);
                }
            }
        }
        __syncthreads();

        auto sym_at = [&](unsigned x) -> uint8_t {
            return all_kept ? symbol_of<MODE>(tb[vlo + x], cls_s) : cc[x];
        };
        // kept symbols of the tile before tile-local byte index i (vlo <= i <= vhi)
        auto kept_before = [&](int i) -> unsigned {
            if (i >= vhi) return K;
            const int v = i >> 4;
            return (unsigned)kpre[v] + __popc((unsigned)kmask[v] & ((1u << (i & 15)) - 1u));
        };

        // boundaries of the tile
        long long rb_lo = 0;
        long long nb;
        if (BSRC == BSRC_LIST) {
            rb_lo = p.tile_rec[t];
            nb = (long long)p.tile_rec[t + 1] - rb_lo;
        } else {
            nb = (long long)NBb + ((p.end_boundary && t == p.n_tiles - 1) ? 1 : 0);
        }
        const long long chunk_byte0 = rel_lo - p.head_pad;  // chunk index of tile byte 0
        // tile-kept position of boundary i (0 <= i < nb)
        auto bnd_kept = [&](long long i) -> unsigned {
            if (BSRC == BSRC_LIST) {
                const long long pos = p.seq_offsets[rb_lo + i] - chunk_byte0;
                return kept_before((int)pos);
            }
            if (i >= NBb) return K;  // end-of-stream boundary
            // select the i-th set bit: last vector with bpre <= i
            int lo = 0, hi = NV - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bpre[mid] <= i) lo = mid; else hi = mid - 1;
            }
            unsigned m = bmask[lo];
            for (unsigned r = (unsigned)(i - bpre[lo]); r > 0; --r) m &= m - 1;
            return kept_before(16 * lo + __ffs(m) - 1);
        };

        // ------------------------------------------ 4. tile scan element
        {
            long long dsum = 0;
            if (nb >= 2) {
                for (long long i = tid; i + 1 < nb; i += NT) {
                    const long long a = bnd_kept(i), b = bnd_kept(i + 1);
                    dsum += (b - a + k - 1) / k;
                }
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
                    const long long first = bnd_kept(0), last = bnd_kept(nb - 1);
                    a.h = first;
                    a.t = K - last;
                    a.d = d + a.t / k;
                    open = a.t;
                }
                unsigned long long codes = 0;
                if (MODE == MODE_KMER && k > 1) {
                    int n = (int)(open < k - 1 ? open : k - 1);
                    unsigned long long bits = 0;
                    for (int q = 0; q < n; ++q)
                        bits |= (unsigned long long)(sym_at(K - 1 - q) & 7) << (3 * q);
                    codes = ((unsigned long long)n << 58) | bits;
                }
                a.codes = codes;
                s_agg = a;
                if (t > 0) {
                    store_agg(&p.desc[t].agg, a);
                    st_release_u32(&p.desc[t].status, ((p.epoch & 0x3fffffffu) << 2) | LB_AGG);
                }
            }
            __syncthreads();
        }
        if (warp == 0) {
            Agg pre = (t == 0) ? carry : lookback_counts(p, t, carry);
            if (lane == 0) {
                const Agg incl = agg_combine(pre, s_agg, k);
                store_agg(&p.desc[t].incl, incl);
                st_release_u32(&p.desc[t].status, ((p.epoch & 0x3fffffffu) << 2) | LB_INCL);
                s_prefix = pre;
                if (t == p.n_tiles - 1) {
                    if (p.totals_out) {
                        p.totals_out[0] = incl.d;
                        p.totals_out[1] = incl.nb > 0 ? incl.nb - 1 : 0;
                    }
                    if (p.carry_out) {
                        Carry c;
                        c.a = incl;
                        c.hstate = (BSRC == BSRC_FASTA) ? s_hend : HS_LS;
                        c.pad = 0;
                        *p.carry_out = c;
                    }
                }
            }
        }
        __syncthreads();
        if (dev_failed(p.status)) break;

        // ------------------------------------------------------- 5. emit
        const Agg P = s_prefix;
        const long long T0 = (P.nb > 0) ? P.d : 0;
        const long long R0 = P.nb;
        const long long J = (P.nb > 0) ? P.t : P.h;

        if (MODE != MODE_KMER || k == 1) {
            // one token per kept symbol
            for (unsigned x = tid; x < K; x += NT) {
                const long long o = T0 + x;
                if (o >= p.out_cap) break;
                const uint8_t s = sym_at(x);
                if (MODE == MODE_SYM) static_cast<uint8_t *>(p.out)[o] = s;
                else if (MODE == MODE_CHAR) static_cast<int *>(p.out)[o] = lut_s[s];
                else static_cast<int *>(p.out)[o] = (s & 4) ? 4 : (s & 3);
            }
            for (long long i = tid; i < nb; i += NT) {
                const long long g = R0 + i;
                if (g < p.offsets_cap) p.offsets_out[g] = T0 + bnd_kept(i);
            }
        } else {
            const long long unk = 1ll << (2 * k);
            const unsigned long long pcodes = P.codes;
            long long tok_base = 0;
            for (long long seg0 = 0; seg0 < nb + 1; seg0 += kSegChunk) {
                const int nseg = (int)((nb + 1 - seg0) < kSegChunk ? (nb + 1 - seg0) : kSegChunk);
                unsigned cnt[1];
                for (int s = tid; s < nseg; s += NT) {
                    const long long gs = seg0 + s;
                    const unsigned ks = (gs == 0) ? 0u : bnd_kept(gs - 1);
                    const unsigned ke = (gs == nb) ? K : bnd_kept(gs);
                    const long long Js = (gs == 0) ? J : 0;
                    const long long L = ke - ks;
                    long long c;
                    if (gs < nb) c = (Js + L + k - 1) / k - Js / k;   // closed record
                    else c = (Js + L) / k - Js / k;                    // still open
                    seg_k[s] = ks;
                    seg_l[s] = (unsigned)L;
                    seg_c[s] = (unsigned)c;
                }
                __syncthreads();
                // exclusive scan of seg_c over nseg entries (chunked by NT)
                {
                    unsigned carry_sum = 0;
                    for (int b0 = 0; b0 < nseg; b0 += NT) {
                        const int s = b0 + tid;
                        unsigned c = (s < nseg) ? seg_c[s] : 0u;
                        unsigned vv[1] = {c}, ex[1];
                        // reuse the vector scan with one value per thread
                        unsigned tot = block_scan_vec<NT, 1>(vv, ex, s_w);
                        if (s < nseg) seg_c[s] = carry_sum + ex[0];
                        carry_sum += tot;
                        __syncthreads();
                    }
                    cnt[0] = carry_sum;
                }
                __syncthreads();
                const unsigned chunk_total = cnt[0];
                // boundary offsets: boundary (seg0 + s - 1) opens segment seg0 + s
                for (int s = tid; s < nseg; s += NT) {
                    const long long gs = seg0 + s;
                    if (gs == 0) continue;
                    const long long g = R0 + gs - 1;
                    if (g < p.offsets_cap) p.offsets_out[g] = T0 + tok_base + seg_c[s];
                }
                // tokens
                for (unsigned u = tid; u < chunk_total; u += NT) {
                    int lo = 0, hi = nseg - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (seg_c[mid] <= u) lo = mid; else hi = mid - 1;
                    }
                    const long long gs = seg0 + lo;
                    const long long Js = (gs == 0) ? J : 0;
                    const long long m = Js / k + (long long)(u - seg_c[lo]);  // token index in record
                    long long id;
                    if ((m + 1) * k > Js + (long long)seg_l[lo]) {
                        id = unk;  // tail of a closed record
                    } else {
                        const long long x0 = (long long)seg_k[lo] - Js + m * k;
                        long long acc = 0;
                        bool n_seen = false;
                        for (int q = 0; q < k; ++q) {
                            const long long x = x0 + q;
                            unsigned s;
                            if (x < 0) s = (unsigned)(pcodes >> (3 * (-x - 1))) & 7u;
                            else s = sym_at((unsigned)x);
                            n_seen |= (s & 4u) != 0;
                            acc = acc * 4 + (s & 3u);
                        }
                        id = n_seen ? unk : acc;
                    }
                    const long long o = T0 + tok_base + u;
                    if (o < p.out_cap) static_cast<int *>(p.out)[o] = (int)id;
                }
                tok_base += chunk_total;
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

}  // namespace dnatok
