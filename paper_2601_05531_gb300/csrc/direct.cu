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
#include "handle.h"
#include "tile_kernel.cuh"

namespace dnatok {

namespace {

constexpr int kDTile = 16384;  // bytes per tile
constexpr int kDThreads = 256;
constexpr int kDVec = kDTile / 16;             // 16-byte vectors per tile
constexpr int kDVpt = kDVec / kDThreads;       // per thread
constexpr int kPlanThreads = 1024;

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
};

// tokens of a record of L kept symbols: ceil(L / k) (L when k = 1)
__device__ __forceinline__ long long rec_tokens(const DirectParams &q, long long L) {
    return q.k == 1 ? L : (long long)__umul64hi((unsigned long long)(L + q.k - 1), q.kinv);
}

__device__ __forceinline__ void raise_gate(const DirectParams &q) {
    if (*(volatile unsigned *)q.gate != q.epoch) *(volatile unsigned *)q.gate = q.epoch;
}

// id offsets from the record lengths; any malformed offset sends the encode
// to the general path (which reports it).
__global__ void __launch_bounds__(kPlanThreads) direct_plan_kernel(DirectParams q) {
    __shared__ long long wsum[kPlanThreads / 32];
    pdl_launch_dependents();  // the direct kernel may start loading its tiles now
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = q.n_seq;
    const long long per = (n + kPlanThreads - 1) / kPlanThreads;
    const long long r0 = tid * per, r1 = (r0 + per < n) ? r0 + per : n;
    long long sum = 0;
    bool bad = false;
    constexpr int kBatch = 8;  // offsets loaded together, then used
    for (long long rb = r0; rb < r1; rb += kBatch) {
        long long v[kBatch + 1];
#pragma unroll
        for (int i = 0; i <= kBatch; ++i) v[i] = (rb + i <= r1) ? q.so[rb + i] : 0;
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
            if (rb + i >= r1) break;
            if (v[i + 1] < v[i]) bad = true;
            sum += rec_tokens(q, v[i + 1] - v[i]);
        }
    }
    if (tid == 0 && (q.so[0] != 0 || q.so[n] != q.n)) bad = true;
    if (__syncthreads_or(bad)) {
        if (tid == 0) raise_gate(q);
        return;
    }
    long long x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    long long pre = 0, total = 0;
    for (int w = 0; w < kPlanThreads / 32; ++w) {
        if (w < warp) pre += wsum[w];
        total += wsum[w];
    }
    long long run = pre + x - sum;
    for (long long r = r0; r < r1; ++r) {
        q.offsets_out[r] = run;
        run += rec_tokens(q, q.so[r + 1] - q.so[r]);
    }
    if (tid == 0) {
        q.offsets_out[n] = total;
        if (q.totals_out) {
            q.totals_out[0] = total;
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
__device__ __forceinline__ unsigned dpack4(unsigned c) {
    const unsigned r = __byte_perm(c, 0, 0x0123);
    const unsigned m = r | (r >> 6);
    return (m & 0xFu) | ((m >> 12) & 0xF0u);
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

// k-mer ids.  Each CTA walks a contiguous range of tiles, loading the next
// tile's vectors while it emits the current one; k-mers whose first byte lies
// in a tile are written by that tile, record batches of 32 flattened so that
// every thread has work even when records are short.
__global__ void __launch_bounds__(kDThreads) direct_kmer_kernel(DirectParams q) {
    __shared__ uint2 PN[kDVec + 1];     // per vector: 2-bit codes (first in the top bits), N flags
    __shared__ long long s_obase[32];   // output index of the batch's first k-mer, per record
    __shared__ int s_ap0[32], s_lim[32], s_pre[33];
    __shared__ long long s_r0, s_next;
    __shared__ int s_more;
    __shared__ int s_stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long lo = q.head_pad, hi = q.head_pad + q.n;      // valid aligned range
    const int k = q.k;
    const unsigned unk = 1u << (2 * k);
    const unsigned nmask = (1u << k) - 1u;
    const long long per = (q.n_tiles + gridDim.x - 1) / gridDim.x;
    const long long t_begin = blockIdx.x * per;
    const long long t_end = (t_begin + per < q.n_tiles) ? t_begin + per : q.n_tiles;
    bool sep = false;
    uint4 cur[kDVpt];
    // tile-relative 32-bit offsets from here on: the tile's own pointer and
    // the number of its bytes that exist are computed once per tile
    auto tile_valid = [&](long long t) -> int {
        const long long v = hi - t * kDTile;
        return v <= 0 ? 0 : (v >= kDTile + 16 ? kDTile + 16 : (int)v);
    };
    auto load_tile = [&](long long t, uint4 *dst) {
        const uint4 *src = reinterpret_cast<const uint4 *>(q.base + t * kDTile) + tid;
        const int nv = tile_valid(t);
#pragma unroll
        for (int i = 0; i < kDVpt; ++i)
            dst[i] = (16 * (i * kDThreads + tid) < nv) ? __ldg(src + i * kDThreads)
                                                        : make_uint4(0u, 0u, 0u, 0u);
    };
    if (t_begin < t_end) load_tile(t_begin, cur);
    for (long long t = t_begin; t < t_end; ++t) {
        const long long A0 = t * kDTile;
        uint4 nxt[kDVpt];
        if (t + 1 < t_end) load_tile(t + 1, nxt);
        const long long x_lo = (A0 > lo ? A0 : lo) - q.head_pad;
        const long long x_hi = ((A0 + kDTile < hi) ? A0 + kDTile : hi) - q.head_pad;
        if (t == t_begin) {
            // the id offsets come from the plan kernel, which may still be
            // running (programmatic launch): wait for it, then see whether it
            // rejected the offsets
            pdl_wait();
            if (tid == 0) s_stop = (*(volatile const unsigned *)q.gate == q.epoch) ? 1 : 0;
            __syncthreads();
            if (s_stop) return;
        }
        if (warp == 0) {
            const long long r0 = warp_rec_search(q.so, q.n_seq, x_lo, lane);
            if (lane == 0) s_r0 = r0;
        }
        {
            const int nv = tile_valid(t);  // bytes of the tile that exist
            const int first = (A0 < lo) ? (int)(lo - A0) : 0;  // the head pad, first tile only
#pragma unroll
            for (int i = 0; i < kDVpt; ++i) {
                const int v = i * kDThreads + tid;
                const Vec16 c = classify16(cur[i]);
                if (c.low) {
                    const int b0 = 16 * v;
                    unsigned m = 0xFFFFu;
                    if (b0 < first) m &= 0xFFFFu << (first - b0 < 16 ? first - b0 : 16);
                    if (b0 + 16 > nv) m &= (nv - b0 <= 0) ? 0u : ((1u << (nv - b0)) - 1u);
                    if (c.low & m) sep = true;
                }
                PN[v] = make_uint2(c.codes, c.nflags);
            }
        }
        if (tid == 0) {  // halo: the first vector of the next tile
            const long long ab = A0 + kDTile;
            if (ab < hi) {
                const Vec16 c = classify16(__ldg(reinterpret_cast<const uint4 *>(q.base + ab)));
                PN[kDVec] = make_uint2(c.codes, c.nflags);
            } else {
                PN[kDVec] = make_uint2(0u, 0u);
            }
        }
        __syncthreads();
        long long r = s_r0;
        const long long shift = q.head_pad - A0;  // input position -> tile offset
        while (true) {
            if (warp == 0) {
                const long long rr = r + lane;
                int cnt = 0;
                if (rr < q.n_seq) {
                    const long long rs = q.so[rr];
                    if (rs < x_hi) {
                        const long long re = q.so[rr + 1];
                        const long long s0 = rs > x_lo ? rs : x_lo;
                        const long long s1 = re < x_hi ? re : x_hi;
                        if (s1 > s0) {
                            const long long m_lo = rec_tokens(q, s0 - rs);
                            cnt = (int)(rec_tokens(q, s1 - rs) - m_lo);
                            s_ap0[lane] = (int)(rs + m_lo * k + shift);
                            const long long re_t = re + shift;
                            s_lim[lane] = re_t > kDTile + 32 ? kDTile + 32 : (int)re_t;
                            s_obase[lane] = q.offsets_out[rr] + m_lo;
                        }
                    }
                }
                int x = cnt;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                s_pre[lane + 1] = x;
                if (lane == 0) {
                    s_pre[0] = 0;
                    const long long nr = r + 32;
                    s_more = (nr < q.n_seq && q.so[nr] < x_hi) ? 1 : 0;
                    s_next = nr;
                }
            }
            __syncthreads();
            const int total = s_pre[32];
            auto kmer_id = [&](int ap, int lim) -> unsigned {
                unsigned id = unk;
                if (ap + k <= lim) {
                    const int wi = ap >> 4, off = ap & 15;
                    const uint2 a = PN[wi], b = PN[wi + 1];
                    const unsigned tw = __funnelshift_l(b.x, a.x, 2 * off);
                    const unsigned nw = a.y | (b.y << 16);
                    if (!((nw >> off) & nmask)) id = tw >> (32 - 2 * k);
                }
                return id;
            };
            if (s_pre[1] == total) {
                // one record holds every k-mer of the batch (the usual case)
                const int ap0 = s_ap0[0], lim = s_lim[0];
                int *o = static_cast<int *>(q.out) + s_obase[0];
                for (int i = tid; i < total; i += kDThreads) o[i] = (int)kmer_id(ap0 + i * k, lim);
            } else {
                for (int f = tid; f < total; f += kDThreads) {
                    int j = 0;  // largest j with s_pre[j] <= f
#pragma unroll
                    for (int b = 16; b > 0; b >>= 1)
                        if (j + b <= 32 && s_pre[j + b] <= f) j += b;
                    const int i = f - s_pre[j];
                    static_cast<int *>(q.out)[s_obase[j] + i] = (int)kmer_id(s_ap0[j] + i * k, s_lim[j]);
                }
            }
            const bool more = s_more != 0;
            r = s_next;
            __syncthreads();
            if (!more) break;
        }
        if (t + 1 < t_end) {
#pragma unroll
            for (int i = 0; i < kDVpt; ++i) cur[i] = nxt[i];
        }
    }
    if (__syncthreads_or(sep) && tid == 0) raise_gate(q);
}

// Single-nucleotide ids / BPE symbols: one output per byte at the byte's own
// position (no separators), streamed with 16-byte loads.
template <int MODE>
__global__ void __launch_bounds__(kDThreads) direct_byte_kernel(DirectParams q) {
    __shared__ int lut_s[256];
    __shared__ int s_stop;
    const int tid = threadIdx.x;
    pdl_wait();
    if (tid == 0) s_stop = (*(volatile const unsigned *)q.gate == q.epoch) ? 1 : 0;
    __syncthreads();
    if (s_stop) return;
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

}  // namespace

bool direct_eligible(int mode, long long n_seq, const int32_t *lut_host) {
    if (n_seq < 1 || n_seq > 65536) return false;
    if (mode == MODE_CHAR) {
        for (int b = 0x21; b < 256; ++b)
            if (lut_host[b] < 0) return false;  // the table drops a byte the direct path keeps
    }
    return mode == MODE_CHAR || mode == MODE_KMER || mode == MODE_SYM;
}

cudaError_t launch_direct(int mode, const uint8_t *bytes, long long n, const long long *so,
                          long long n_seq, void *out, long long *offsets_out,
                          long long *totals_out, unsigned *gate, unsigned epoch, int k,
                          const int *lut, int sm_count, cudaStream_t s) {
    DirectParams q;
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
    q.n_tiles = (q.head_pad + n + kDTile - 1) / kDTile;
    direct_plan_kernel<<<1, kPlanThreads, 0, s>>>(q);
    if (n > 0) {
        long long grid = (long long)sm_count * 8;
        if (grid > q.n_tiles) grid = q.n_tiles;
        // programmatic dependent launch: it starts while the plan runs
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(kDThreads);
        cfg.stream = s;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr.val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        if (mode == MODE_KMER) {
            cfg.gridDim = dim3((unsigned)grid);
            return cudaLaunchKernelEx(&cfg, direct_kmer_kernel, q);
        }
        long long g2 = ((q.head_pad + n + 15) / 16 + kDThreads - 1) / kDThreads;
        if (g2 > (long long)sm_count * 8) g2 = (long long)sm_count * 8;
        cfg.gridDim = dim3((unsigned)g2);
        if (mode == MODE_CHAR) return cudaLaunchKernelEx(&cfg, direct_byte_kernel<MODE_CHAR>, q);
        return cudaLaunchKernelEx(&cfg, direct_byte_kernel<MODE_SYM>, q);
    }
    return cudaGetLastError();
}

}  // namespace dnatok
