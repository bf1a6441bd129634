// decode.cu -- token ids back to text on the device (Sec. 4, "Decode
// Operations", future work there): a reverse lookup from each id to the
// bases it stands for, run as table gathers like the encode.
//
// Per mode the text of an id is
//   DNATOK_CHAR          one byte: the first byte b with lut[b] == id in the
//                        order "ACGTN", 'A'..'Z', 'a'..'z', 0..255;
//   DNATOK_KMER          k bases for id < 4^k, '?' for UNK = 4^k;
//   DNATOK_KMER_OVERLAP  per record, the first token as DNATOK_KMER and each
//                        later one its last base ('?' for UNK);
//   DNATOK_BPE           the bases the merge table expands it to, N for N_ID;
//   DNATOK_KMER_TABLE    the k digits ("ACGTN") of the smallest window index
//                        whose kmer_lut entry is the id, else the symbol of
//                        the smallest digit whose base id it is.
// CHAR, BPE and KMER_TABLE go through a table built on the host at the first
// call (offsets + text, one entry per id); the k-mer modes are arithmetic.
// An id with no text is counted and writes nothing.
//
// Three launches: dec_tile_kernel<false> (per tile of 2048 ids, its byte
// count and its count of ids without text), tile_scan_kernel (exclusive scan
// of the tile counts, totals), dec_tile_kernel<true> (recount, scan inside the
// block, write the bytes and the record offsets of records starting here).
// The emit assembles a tile's text in shared memory when it fits (16 KB: up
// to 8 bases per id on average) and writes it out in aligned 16-byte stores;
// larger tiles write byte by byte.
#include <cstring>
#include <string>
#include <vector>

#include "handle.h"
#include "search.cuh"

namespace {

using namespace dnatok;

constexpr int kDT = 2048;       // ids per tile
constexpr int kDThreads = 256;  // eight consecutive ids per thread
constexpr int kDOut = 16384;    // text bytes of a tile staged in shared memory
constexpr int kDPer = kDT / kDThreads;

enum { DEC_TABLE = 0, DEC_KMER = 1, DEC_OVL = 2 };

struct DecArgs {
    const int *ids;
    long long n_ids;
    const long long *keys;  // id_offsets (n_rec + 1)
    long long n_rec;
    const int *off;          // DEC_TABLE: text offsets (V + 1)
    const uint8_t *text;
    long long V;
    int k;
    long long *tsum, *tinv;
    uint8_t *out;
    long long cap;
    long long *rec_out;
};

// "ACGT"[c] for c in 0..3
__device__ __forceinline__ uint8_t base_char(int c) { return (uint8_t)(0x54474341u >> (8 * c)); }

template <int MODE>
__device__ __forceinline__ int dec_len(const DecArgs &a, int v, bool first) {
    if (MODE == DEC_TABLE) return (v >= 0 && v < a.V) ? __ldg(a.off + v + 1) - __ldg(a.off + v) : 0;
    const int unk = 1 << (2 * a.k);
    if (MODE == DEC_OVL && !first) return (v >= 0 && v <= unk) ? 1 : 0;
    if (v >= 0 && v < unk) return a.k;
    return v == unk ? 1 : 0;
}

template <int MODE, bool EMIT>
__global__ void __launch_bounds__(kDThreads) dec_tile_kernel(DecArgs a) {
    __shared__ uint8_t s_first[kDT];
    __shared__ int s_pos[kDT];
    __shared__ __align__(16) uint8_t s_out[kDOut + 32];
    __shared__ long long s_ra, s_rb;
    __shared__ int s_wsum[kDThreads / 32], s_winv[kDThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n_tiles = (a.n_ids + kDT - 1) / kDT;
    // a contiguous run of tiles per CTA: the records starting in one tile
    // begin where the previous tile's ended
    const long long t_begin = (long long)blockIdx.x * n_tiles / gridDim.x;
    const long long t_end = (long long)(blockIdx.x + 1) * n_tiles / gridDim.x;
    for (long long tile = t_begin; tile < t_end; ++tile) {
        const long long t0 = tile * kDT;
        const long long t1 = (t0 + kDT < a.n_ids) ? t0 + kDT : a.n_ids;
        const bool need_rec = (MODE == DEC_OVL) || EMIT;
        if (need_rec) {
            // the records starting in [t0, t1): [s_ra, s_rb)
            if (tile == t_begin) {
                if (warp == 0) {
                    const long long r = warp_first_ge(a.keys, a.n_rec, t0);
                    if (lane == 0) s_ra = r < a.n_rec ? r : a.n_rec;
                }
                __syncthreads();
            } else if (tid == 0) {
                s_ra = s_rb;
            }
            if (warp == 0) {
                // forward from s_ra, 32 offsets per round (offsets are sorted)
                long long r = (tile == t_begin) ? s_ra : s_rb;
                while (true) {
                    const long long idx = r + lane;
                    const unsigned m = __ballot_sync(0xffffffffu, idx <= a.n_rec && a.keys[idx] < t1);
                    const int c = __popc(m);
                    r += c;
                    if (c < 32) break;
                }
                __syncwarp();
                if (lane == 0) s_rb = r;
            }
            if (MODE == DEC_OVL)
                for (int i = tid; i < kDT; i += kDThreads) s_first[i] = 0;
            __syncthreads();
            if (MODE == DEC_OVL)
                for (long long r = s_ra + tid; r < s_rb; r += kDThreads) {
                    const long long f = a.keys[r] - t0;
                    if (f >= 0 && f < kDT) s_first[f] = 1;
                }
            __syncthreads();
        }
        int v[kDPer], len[kDPer], sum = 0, bad = 0;
#pragma unroll
        for (int q = 0; q < kDPer; ++q) {
            const long long t = t0 + (long long)tid * kDPer + q;
            v[q] = 0;
            len[q] = 0;
            if (t >= t1) continue;
            v[q] = __ldg(a.ids + t);
            len[q] = dec_len<MODE>(a, v[q], MODE == DEC_OVL && s_first[t - t0]);
            sum += len[q];
            bad += len[q] == 0;
        }
        int x = sum, y = bad;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int p = __shfl_up_sync(0xffffffffu, x, o);
            const int c = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) {
                x += p;
                y += c;
            }
        }
        if (lane == 31) {
            s_wsum[warp] = x;
            s_winv[warp] = y;
        }
        __syncthreads();
        if (!EMIT) {
            if (tid == 0) {
                long long tt = 0, ti = 0;
                for (int w = 0; w < kDThreads / 32; ++w) {
                    tt += s_wsum[w];
                    ti += s_winv[w];
                }
                a.tsum[tile] = tt;
                a.tinv[tile] = ti;
            }
        } else {
            int local = x - sum, total = 0;
            for (int w = 0; w < kDThreads / 32; ++w) {
                if (w < warp) local += s_wsum[w];
                total += s_wsum[w];
            }
            const long long base = a.tsum[tile];
            // staged: the text goes to s_out[shift + local], shift being the
            // misalignment of its global start, then out in aligned chunks
            const int shift = (int)(reinterpret_cast<uintptr_t>(a.out + base) & 15u);
            const bool staged = total + shift <= kDOut;
#pragma unroll
            for (int q = 0; q < kDPer; ++q) {
                s_pos[tid * kDPer + q] = local;
                const long long p = base + local;
                uint8_t *dst = staged ? s_out + shift + local : a.out + p;
                if (len[q] > 0 && (staged || p + len[q] <= a.cap)) {
                    if (MODE == DEC_TABLE) {
                        const int o = __ldg(a.off + v[q]);
                        for (int i = 0; i < len[q]; ++i) dst[i] = __ldg(a.text + o + i);
                    } else if (len[q] == 1) {
                        const int unk = 1 << (2 * a.k);
                        dst[0] = v[q] == unk ? (uint8_t)'?' : base_char(v[q] & 3);
                    } else {
                        for (int i = 0; i < a.k; ++i)
                            dst[i] = base_char((v[q] >> (2 * (a.k - 1 - i))) & 3);
                    }
                }
                local += len[q];
            }
            __syncthreads();
            if (staged) {
                const int span = shift + total;
                uint8_t *g = a.out + (base - shift);  // 16-byte aligned
                const long long lim = a.cap - (base - shift);  // bytes of g inside the buffer
                for (int c = tid; c < (span + 15) >> 4; c += kDThreads) {
                    const int lo = c * 16, hi = lo + 16;
                    if (lo >= shift && hi <= span && hi <= lim) {
                        *reinterpret_cast<uint4 *>(g + lo) = *reinterpret_cast<const uint4 *>(s_out + lo);
                    } else {
                        for (int y = lo > shift ? lo : shift; y < (hi < span ? hi : span); ++y)
                            if (y < lim) g[y] = s_out[y];
                    }
                }
            }
            for (long long r = s_ra + tid; r < s_rb; r += kDThreads) {
                const long long f = a.keys[r] - t0;
                if (f >= 0 && f < t1 - t0) a.rec_out[r] = base + s_pos[f];
            }
        }
        __syncthreads();  // shared memory is reused by the next tile
    }
}

template <int MODE>
cudaError_t launch_dec(bool emit, unsigned grid, const DecArgs &a, cudaStream_t s) {
    if (emit) dec_tile_kernel<MODE, true><<<grid, kDThreads, 0, s>>>(a);
    else dec_tile_kernel<MODE, false><<<grid, kDThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// The text of every id on the host: offsets (V + 1) and bytes.
dnatok_status build_text(dnatok_handle *h, std::vector<int32_t> &off, std::string &text) {
    constexpr long long kMaxV = 1ll << 24;
    constexpr long long kMaxText = 256ll << 20;
    std::vector<std::string> tok;
    if (h->mode == DNATOK_CHAR) {
        long long V = 0;
        for (int b = 0; b < 256; ++b)
            if (h->lut_host[b] >= 0 && h->lut_host[b] + 1ll > V) V = h->lut_host[b] + 1ll;
        if (V > kMaxV) return fail(h, DNATOK_ERR_TABLE, "decode: table ids above 2^24");
        tok.assign((size_t)V, std::string());
        std::vector<int> order;
        for (const char *c = "ACGTN"; *c; ++c) order.push_back((unsigned char)*c);
        for (int c = 'A'; c <= 'Z'; ++c) order.push_back(c);
        for (int c = 'a'; c <= 'z'; ++c) order.push_back(c);
        for (int c = 0; c < 256; ++c) order.push_back(c);
        for (int b : order) {
            const int v = h->lut_host[b];
            if (v >= 0 && tok[(size_t)v].empty()) tok[(size_t)v] = std::string(1, (char)b);
        }
    } else if (h->mode == DNATOK_BPE) {
        const long long M = (long long)h->merges_host.size() / 2;
        tok.assign((size_t)(5 + M), std::string());
        for (int c = 0; c < 4; ++c) tok[(size_t)c] = std::string(1, "ACGT"[c]);
        long long total = 5;
        for (long long r = 0; r < M; ++r) {
            const int l = h->merges_host[2 * r], q = h->merges_host[2 * r + 1];
            total += (long long)tok[(size_t)l].size() + (long long)tok[(size_t)q].size();
            if (total > kMaxText) return fail(h, DNATOK_ERR_TABLE, "decode: BPE text above 256 MB");
            tok[(size_t)(4 + r)] = tok[(size_t)l] + tok[(size_t)q];
        }
        tok[(size_t)(4 + M)] = "N";
    } else if (h->mode == DNATOK_KMER_TABLE) {
        long long V = 0;
        for (int32_t v : h->klut_host)
            if (v + 1ll > V) V = v + 1ll;
        for (int d = 0; d < 5; ++d)
            if (h->base_ids[d] + 1ll > V) V = h->base_ids[d] + 1ll;
        if (V > kMaxV) return fail(h, DNATOK_ERR_TABLE, "decode: table ids above 2^24");
        tok.assign((size_t)V, std::string());
        const int k = h->k;
        for (size_t index = 0; index < h->klut_host.size(); ++index) {
            const int v = h->klut_host[index];
            if (v < 0 || !tok[(size_t)v].empty()) continue;
            std::string t((size_t)k, 'A');
            size_t x = index;
            for (int i = k - 1; i >= 0; --i) {
                t[(size_t)i] = "ACGTN"[x % 5];
                x /= 5;
            }
            tok[(size_t)v] = t;
        }
        for (int d = 0; d < 5; ++d)
            if (tok[(size_t)h->base_ids[d]].empty()) tok[(size_t)h->base_ids[d]] = std::string(1, "ACGTN"[d]);
    }
    off.assign(tok.size() + 1, 0);
    text.clear();
    int lmax = 1;
    for (size_t v = 0; v < tok.size(); ++v) {
        text += tok[v];
        off[v + 1] = (int32_t)text.size();
        if ((int)tok[v].size() > lmax) lmax = (int)tok[v].size();
    }
    h->dec_max_len = lmax;
    return DNATOK_OK;
}

dnatok_status ensure_tables(dnatok_handle *h) {
    if (h->dec_v >= 0) return DNATOK_OK;
    if (h->mode == DNATOK_KMER || h->mode == DNATOK_KMER_OVERLAP) {
        h->dec_v = 0;
        h->dec_max_len = h->k;
        return DNATOK_OK;
    }
    std::vector<int32_t> off;
    std::string text;
    dnatok_status st = build_text(h, off, text);
    if (st != DNATOK_OK) return st;
    cudaError_t e = cudaMalloc(&h->d_dec_off, sizeof(int32_t) * off.size());
    if (e == cudaSuccess) e = cudaMalloc(&h->d_dec_text, text.size() + 1);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_dec_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !text.empty())
        e = cudaMemcpy(h->d_dec_text, text.data(), text.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(h->d_dec_off);
        cudaFree(h->d_dec_text);
        h->d_dec_off = nullptr;
        h->d_dec_text = nullptr;
        return fail_cuda(h, e, "decode table upload");
    }
    h->dec_v = (long long)off.size() - 1;
    return DNATOK_OK;
}

}  // namespace

namespace dnatok {

void dec_destroy(dnatok_handle *h) {
    cudaFree(h->d_dec_off);
    cudaFree(h->d_dec_text);
    cudaFree(h->d_dsum);
    cudaFree(h->d_dinv);
    h->d_dec_off = nullptr;
    h->d_dec_text = nullptr;
    h->d_dsum = h->d_dinv = nullptr;
    h->dsum_cap = 0;
    h->dec_v = -1;
}

}  // namespace dnatok

extern "C" {

dnatok_status dnatok_max_decoded_bytes(dnatok_handle *h, int64_t n_ids, int64_t n_seq,
                                       int64_t *cap) {
    if (!h || !cap || n_ids < 0 || n_seq < 0) return DNATOK_ERR_ARG;
    dnatok_status st = ensure_tables(h);
    if (st != DNATOK_OK) return st;
    if (h->mode == DNATOK_KMER_OVERLAP)
        *cap = n_ids + (n_seq < n_ids ? n_seq : n_ids) * (int64_t)(h->k - 1);
    else
        *cap = n_ids * (int64_t)h->dec_max_len;
    return DNATOK_OK;
}

dnatok_status dnatok_decode(dnatok_handle *h, const int32_t *ids_d, int64_t n_ids,
                            const int64_t *id_offsets_d, int64_t n_seq, uint8_t *bytes_out_d,
                            int64_t bytes_capacity, int64_t *byte_offsets_d, int64_t *totals_d,
                            dnatok_cuda_stream stream) {
    if (!h) return DNATOK_ERR_ARG;
    if (n_ids < 0 || n_seq < 0 || (n_ids > 0 && !ids_d) || !id_offsets_d || !byte_offsets_d)
        return fail(h, DNATOK_ERR_ARG, "bad decode arguments");
    if (((uintptr_t)id_offsets_d | (uintptr_t)byte_offsets_d | (uintptr_t)totals_d) & 7u)
        return fail(h, DNATOK_ERR_ARG, "int64 arrays must be 8-byte aligned");
    if ((uintptr_t)ids_d & 3u) return fail(h, DNATOK_ERR_ARG, "ids must be 4-byte aligned");
    int64_t need = 0;
    dnatok_status st = dnatok_max_decoded_bytes(h, n_ids, n_seq, &need);
    if (st != DNATOK_OK) return st;
    if (bytes_capacity < need || (need > 0 && !bytes_out_d))
        return fail(h, DNATOK_ERR_CAPACITY, "bytes_out smaller than dnatok_max_decoded_bytes()");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long long n_tiles = (n_ids + kDT - 1) / kDT;
    if (n_tiles + 1 > h->dsum_cap) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            return fail(h, DNATOK_ERR_STATE, "decode workspace must grow during stream capture");
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaStreamSynchronize");
        cudaFree(h->d_dsum);
        cudaFree(h->d_dinv);
        h->d_dsum = h->d_dinv = nullptr;
        h->dsum_cap = 0;
        const long long c = n_tiles + n_tiles / 8 + 16;
        e = cudaMalloc(&h->d_dsum, sizeof(long long) * (size_t)c);
        if (e == cudaSuccess) e = cudaMalloc(&h->d_dinv, sizeof(long long) * (size_t)c);
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMalloc(decode workspace)");
        h->dsum_cap = c;
    }
    DecArgs a;
    a.ids = ids_d;
    a.n_ids = n_ids;
    a.keys = reinterpret_cast<const long long *>(id_offsets_d);
    a.n_rec = n_seq;
    a.off = h->d_dec_off;
    a.text = h->d_dec_text;
    a.V = h->dec_v;
    a.k = h->k;
    a.tsum = h->d_dsum;
    a.tinv = h->d_dinv;
    a.out = bytes_out_d;
    a.cap = bytes_capacity;
    a.rec_out = reinterpret_cast<long long *>(byte_offsets_d);
    long long grid = (long long)h->sm_count * 8;
    if (grid > n_tiles) grid = n_tiles;
    if (grid < 1) grid = 1;
    const int mode = (h->mode == DNATOK_KMER) ? DEC_KMER
                     : (h->mode == DNATOK_KMER_OVERLAP) ? DEC_OVL : DEC_TABLE;
    for (int pass = 0; pass < 2; ++pass) {
        cudaError_t e;
        if (pass == 1) {
            tile_scan_kernel<<<1, kTileScanThreads, 0, s>>>(
                h->d_dsum, h->d_dinv, a.keys, nullptr, n_seq, nullptr, n_ids, kDT, a.rec_out,
                reinterpret_cast<long long *>(totals_d), nullptr, nullptr, 0u, false);
            e = cudaGetLastError();
            if (e != cudaSuccess) return fail_cuda(h, e, "decode scan launch");
        }
        if (mode == DEC_KMER) e = launch_dec<DEC_KMER>(pass == 1, (unsigned)grid, a, s);
        else if (mode == DEC_OVL) e = launch_dec<DEC_OVL>(pass == 1, (unsigned)grid, a, s);
        else e = launch_dec<DEC_TABLE>(pass == 1, (unsigned)grid, a, s);
        if (e != cudaSuccess) return fail_cuda(h, e, "decode launch");
    }
    return DNATOK_OK;
}

}  // extern "C"
