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
    const int *lut;            // MODE_CHAR
    long long n_tiles;
};

__device__ __forceinline__ void raise_gate(const DirectParams &q) {
    if (*(volatile unsigned *)q.gate != q.epoch) *(volatile unsigned *)q.gate = q.epoch;
}

// id offsets from the record lengths; any malformed offset sends the encode
// to the general path (which reports it).
__global__ void __launch_bounds__(kPlanThreads) direct_plan_kernel(DirectParams q) {
    __shared__ long long wsum[kPlanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = q.n_seq;
    const long long per = (n + kPlanThreads - 1) / kPlanThreads;
    const long long r0 = tid * per, r1 = (r0 + per < n) ? r0 + per : n;
    long long sum = 0;
    bool bad = false;
    for (long long r = r0; r < r1; ++r) {
        const long long a = q.so[r], b = q.so[r + 1];
        if (b < a) bad = true;
        const long long L = b - a;
        sum += (q.k > 1) ? (L + q.k - 1) / q.k : L;
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
        const long long L = q.so[r + 1] - q.so[r];
        run += (q.k > 1) ? (L + q.k - 1) / q.k : L;
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

template <int MODE>
__global__ void __launch_bounds__(kDThreads) direct_kernel(DirectParams q) {
    __shared__ unsigned P[kDVec + 1];        // 2-bit codes, 16 per word, first in the top bits
    __shared__ unsigned NB[kDVec + 1];       // N flags, byte j in bit j
    __shared__ int lut_s[256];
    const int tid = threadIdx.x;
    // the plan found the offsets malformed: the general path takes over (and
    // the ids positions below would not be trustworthy)
    if (*(volatile const unsigned *)q.gate == q.epoch) return;
    if (MODE == MODE_CHAR) {
        for (int i = tid; i < 256; i += kDThreads) lut_s[i] = q.lut[i];
        __syncthreads();
    }
    const long long lo = q.head_pad, hi = q.head_pad + q.n;  // valid aligned range
    bool sep = false;
    for (long long t = blockIdx.x; t < q.n_tiles; t += gridDim.x) {
        const long long A0 = t * kDTile;
#pragma unroll
        for (int i = 0; i < kDVpt; ++i) {
            const int v = i * kDThreads + tid;
            const long long ab = A0 + 16ll * v;
            if (ab >= hi) {
                if (MODE == MODE_KMER) {
                    P[v] = 0u;
                    NB[v] = 0u;
                }
                continue;
            }
            const uint4 w = __ldg(reinterpret_cast<const uint4 *>(q.base + ab));
            const unsigned m = lane_mask16(ab, lo, hi);
            const unsigned c0 = dcodes4(w.x), c1 = dcodes4(w.y), c2 = dcodes4(w.z), c3 = dcodes4(w.w);
            const unsigned l16 = dgather4(dlow4(w.x)) | (dgather4(dlow4(w.y)) << 4) |
                                 (dgather4(dlow4(w.z)) << 8) | (dgather4(dlow4(w.w)) << 12);
            if (l16 & m) sep = true;
            const unsigned n16 = dgather4(dnonbase4(w.x, c0)) | (dgather4(dnonbase4(w.y, c1)) << 4) |
                                 (dgather4(dnonbase4(w.z, c2)) << 8) |
                                 (dgather4(dnonbase4(w.w, c3)) << 12);
            if (MODE == MODE_KMER) {
                P[v] = (dpack4(c0) << 24) | (dpack4(c1) << 16) | (dpack4(c2) << 8) | dpack4(c3);
                NB[v] = n16;
            } else {
                // one id per byte, at the byte's own position (no separators)
                const long long x0 = ab - q.head_pad;
                const unsigned cw[4] = {c0, c1, c2, c3};
                const unsigned bw[4] = {w.x, w.y, w.z, w.w};
                if (MODE == MODE_SYM) {
                    unsigned o[4];
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        unsigned nb = (n16 >> (4 * g)) & 0xFu;
                        unsigned s4 = cw[g];
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            if ((nb >> b) & 1u) s4 = (s4 & ~(0xFFu << (8 * b))) | (4u << (8 * b));
                        o[g] = s4;
                    }
                    uint8_t *out = static_cast<uint8_t *>(q.out);
                    if (m == 0xFFFFu && q.head_pad == 0) {
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
                    if (m == 0xFFFFu && q.head_pad == 0) {
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
        }
        if (MODE != MODE_KMER) continue;
        // halo: the vector after the tile, for k-mers that start near its end
        if (tid == 0) {
            const long long ab = A0 + kDTile;
            if (ab < hi) {
                const uint4 w = __ldg(reinterpret_cast<const uint4 *>(q.base + ab));
                const unsigned c0 = dcodes4(w.x), c1 = dcodes4(w.y), c2 = dcodes4(w.z), c3 = dcodes4(w.w);
                P[kDVec] = (dpack4(c0) << 24) | (dpack4(c1) << 16) | (dpack4(c2) << 8) | dpack4(c3);
                NB[kDVec] = dgather4(dnonbase4(w.x, c0)) | (dgather4(dnonbase4(w.y, c1)) << 4) |
                            (dgather4(dnonbase4(w.z, c2)) << 8) | (dgather4(dnonbase4(w.w, c3)) << 12);
            } else {
                P[kDVec] = 0u;
                NB[kDVec] = 0u;
            }
        }
        __syncthreads();
        // k-mers whose first byte lies in this tile, record by record
        const int k = q.k;
        const unsigned unk = 1u << (2 * k);
        const unsigned long long kmask = (1ull << (2 * k)) - 1ull;
        const long long x_lo = (A0 > lo ? A0 : lo) - q.head_pad;
        const long long x_hi = ((A0 + kDTile < hi) ? A0 + kDTile : hi) - q.head_pad;
        if (x_lo < x_hi) {
            // last record starting at or before x_lo
            long long a = 0, b = q.n_seq;  // so[a] <= x_lo
            while (a < b) {
                const long long mid = (a + b + 1) >> 1;
                if (q.so[mid] <= x_lo) a = mid;
                else b = mid - 1;
            }
            int *out = static_cast<int *>(q.out);
            for (long long r = a; r < q.n_seq; ++r) {
                const long long rs = q.so[r], re = q.so[r + 1];
                if (rs >= x_hi) break;
                if (re <= x_lo || re == rs) continue;
                const long long s0 = rs > x_lo ? rs : x_lo;
                const long long s1 = re < x_hi ? re : x_hi;
                const long long m_lo = (s0 - rs + k - 1) / k;
                const long long m_hi = (s1 - rs + k - 1) / k;
                const long long base = q.offsets_out[r];
                for (long long mm = m_lo + tid; mm < m_hi; mm += kDThreads) {
                    const long long p = rs + mm * k;
                    unsigned id = unk;
                    if (p + k <= re) {
                        const int ap = (int)(p + q.head_pad - A0);  // 0 .. kDTile - 1
                        const int wi = ap >> 4, off = ap & 15;
                        const unsigned long long win = ((unsigned long long)P[wi] << 32) | P[wi + 1];
                        const unsigned code = (unsigned)((win >> (64 - 2 * (off + k))) & kmask);
                        const unsigned nwin = NB[wi] | (NB[wi + 1] << 16);
                        if (!((nwin >> off) & ((1u << k) - 1u))) id = code;
                    }
                    out[base + mm] = (int)id;
                }
            }
        }
        __syncthreads();
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
    q.lut = lut;
    q.n_tiles = (q.head_pad + n + kDTile - 1) / kDTile;
    direct_plan_kernel<<<1, kPlanThreads, 0, s>>>(q);
    if (n > 0) {
        long long grid = (long long)sm_count * 8;
        if (grid > q.n_tiles) grid = q.n_tiles;
        if (mode == MODE_KMER) direct_kernel<MODE_KMER><<<(unsigned)grid, kDThreads, 0, s>>>(q);
        else if (mode == MODE_CHAR) direct_kernel<MODE_CHAR><<<(unsigned)grid, kDThreads, 0, s>>>(q);
        else direct_kernel<MODE_SYM><<<(unsigned)grid, kDThreads, 0, s>>>(q);
    }
    return cudaGetLastError();
}

}  // namespace dnatok
