// feed.cu -- what sits around the encode on its way to a model, all on the
// device and without a handle:
//   * the fixed-shape model feed (Algorithm 2: rows left-padded with id_pad
//     to token_len, their own tokens right-aligned; Sec. 2.2: int32 ids
//     promoted to int64 on the device), one-shot or micro-batched over two
//     streams with two buffers used in turn (Sec. 2.2, "Pipelined streaming");
//   * the reverse complement of every record (Sec. 4, "Integration with Data
//     Augmentation": the augmentation the paper leaves to future GPU work).
#include <cuda_runtime.h>

#include <cstdint>

#include "dnatok.h"
#include "search.cuh"

namespace {

// ------------------------------------------------------------------- feed

constexpr int kFThreads = 256;
constexpr int kFStrip = 1024;       // columns per CTA of the long-row kernel
constexpr int kFShortRows = 8;      // rows per CTA (one per warp) of the short-row kernel
constexpr long long kFShort = 512;  // rows up to this length take the short-row kernel

// Row i, column c: id_pad before the row's tokens, then its first
// min(m, token_len) ids.
template <typename T>
__device__ __forceinline__ T feed_value(const int *ids, long long o0, long long m, long long L,
                                        long long c, T pad) {
    const long long mm = m < L ? m : L;
    const long long lead = L - mm;
    return c < lead ? pad : (T)__ldg(ids + o0 + (c - lead));
}

// long rows: CTA (row, strip of 1024 columns), four columns per thread,
// consecutive threads on consecutive columns
template <typename T>
__global__ void __launch_bounds__(kFThreads) feed_long_kernel(const int *ids, const long long *offs,
                                                              long long row0, long long L, T pad,
                                                              long long strips, T *out) {
    const long long row = blockIdx.x / strips;
    const long long strip = blockIdx.x % strips;
    const long long o0 = offs[row0 + row], m = offs[row0 + row + 1] - o0;
    T *dst = out + row * L;
#pragma unroll
    for (int q = 0; q < kFStrip / kFThreads; ++q) {
        const long long c = strip * kFStrip + q * kFThreads + threadIdx.x;
        if (c < L) dst[c] = feed_value<T>(ids, o0, m, L, c, pad);
    }
}

// short rows: one warp per row, lanes stride the row
template <typename T>
__global__ void __launch_bounds__(kFThreads) feed_short_kernel(const int *ids, const long long *offs,
                                                               long long row0, long long n_rows,
                                                               long long L, T pad, T *out) {
    const long long row = (long long)blockIdx.x * kFShortRows + (threadIdx.x >> 5);
    if (row >= n_rows) return;
    const long long o0 = offs[row0 + row], m = offs[row0 + row + 1] - o0;
    T *dst = out + row * L;
    for (long long c = threadIdx.x & 31; c < L; c += 32) dst[c] = feed_value<T>(ids, o0, m, L, c, pad);
}

template <typename T>
cudaError_t launch_feed(const int *ids, const long long *offs, long long row0, long long n_rows,
                        long long L, long long pad, void *out, cudaStream_t s) {
    if (n_rows == 0 || L == 0) return cudaSuccess;
    T *o = static_cast<T *>(out);
    if (L <= kFShort) {
        const long long grid = (n_rows + kFShortRows - 1) / kFShortRows;
        feed_short_kernel<T><<<(unsigned)grid, kFThreads, 0, s>>>(ids, offs, row0, n_rows, L, (T)pad, o);
    } else {
        const long long strips = (L + kFStrip - 1) / kFStrip;
        feed_long_kernel<T><<<(unsigned)(n_rows * strips), kFThreads, 0, s>>>(ids, offs, row0, L,
                                                                              (T)pad, strips, o);
    }
    return cudaGetLastError();
}

dnatok_status feed_args_ok(const int32_t *ids_d, const int64_t *id_offsets_d, int64_t row_begin,
                           int64_t n_rows, int64_t token_len, int64_t id_pad, int32_t out_bytes) {
    if (!id_offsets_d || row_begin < 0 || n_rows < 0 || token_len < 0) return DNATOK_ERR_ARG;
    if (out_bytes != 4 && out_bytes != 8) return DNATOK_ERR_ARG;
    if (out_bytes == 4 && (id_pad < INT32_MIN || id_pad > INT32_MAX)) return DNATOK_ERR_ARG;
    if (((uintptr_t)id_offsets_d & 7u) || ((uintptr_t)ids_d & 3u)) return DNATOK_ERR_ARG;
    // grid limits: rows x strips below 2^31
    const long long strips = (token_len + kFStrip - 1) / kFStrip;
    if (n_rows > 0 && (token_len > kFShort ? n_rows * strips : n_rows / kFShortRows) >= (1ll << 31))
        return DNATOK_ERR_ARG;
    return DNATOK_OK;
}

// ------------------------------------------------------ reverse complement

constexpr int kRThreads = 256;
constexpr int kRStep = 512;  // bytes per warp step, 16 per lane

__device__ __forceinline__ uint8_t comp_of(int b) {
    switch (b) {
        case 'A': return 'T'; case 'T': return 'A'; case 'C': return 'G'; case 'G': return 'C';
        case 'R': return 'Y'; case 'Y': return 'R'; case 'K': return 'M'; case 'M': return 'K';
        case 'B': return 'V'; case 'V': return 'B'; case 'D': return 'H'; case 'H': return 'D';
        case 'a': return 't'; case 't': return 'a'; case 'c': return 'g'; case 'g': return 'c';
        case 'r': return 'y'; case 'y': return 'r'; case 'k': return 'm'; case 'm': return 'k';
        case 'b': return 'v'; case 'v': return 'b'; case 'd': return 'h'; case 'h': return 'd';
        default: return (uint8_t)b;
    }
}

// Warp-streamed: each warp owns the output range [B0, B1) (B0 a multiple of
// 512) and walks it in 512-byte steps, lane l writing the 16 bytes
// [p, p + 16), p = step + 16 l.  The record [s, e) of the step is kept in
// registers (the same in every lane) and looked up again, by a one-warp
// search, only when a step starts past it.  A chunk inside the record with a
// 16-byte aligned output takes the fast path: the 16 mirrored input bytes
// come from four or five aligned words, are shifted into place, reversed
// and complemented through a shared table, and leave in one 16-byte store.
// Other chunks (record boundaries, the end, unaligned output) go byte by
// byte.  No block-wide barrier after the table is built.
__global__ void __launch_bounds__(kRThreads) revcomp_kernel(const uint8_t *__restrict__ in,
                                                            long long n,
                                                            const long long *__restrict__ so,
                                                            long long n_seq,
                                                            uint8_t *__restrict__ out, int vec_out,
                                                            long long per_warp) {
    __shared__ uint8_t s_comp[256];
    const int tid = threadIdx.x, lane = tid & 31;
    s_comp[tid] = comp_of(tid);
    __syncthreads();
    const long long gw = ((long long)blockIdx.x * kRThreads + tid) >> 5;
    const long long B0 = gw * per_warp;
    if (B0 >= n) return;
    const long long B1 = (B0 + per_warp < n) ? B0 + per_warp : n;
    long long r = dnatok::warp_find_le(so, n_seq, B0);
    long long s = so[r], e = so[r + 1];
    for (long long p0 = B0; p0 < B1; p0 += kRStep) {
        const long long p = p0 + 16 * lane;
        if (vec_out && p < B1 && p >= s && p + 16 <= e && s >= 0 && e <= n) {
            // input bytes [a, a + 16) mirror output bytes [p, p + 16)
            const uintptr_t ua = reinterpret_cast<uintptr_t>(in + (s + e - p - 16));
            const unsigned *wp = reinterpret_cast<const unsigned *>(ua & ~(uintptr_t)3);
            const unsigned sh = (unsigned)(ua & 3) * 8u;
            unsigned w[5];
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = __ldg(wp + i);
            // the fifth word holds input bytes only when the start is unaligned
            w[4] = sh ? __ldg(wp + 4) : 0u;
            uint4 v;
            unsigned *vv = reinterpret_cast<unsigned *>(&v);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // output word j = input bytes 4(3-j) .. 4(3-j)+3, reversed
                const unsigned y = __funnelshift_r(w[3 - j], w[4 - j], sh);
                vv[j] = (unsigned)s_comp[y >> 24] | ((unsigned)s_comp[(y >> 16) & 0xFFu] << 8) |
                        ((unsigned)s_comp[(y >> 8) & 0xFFu] << 16) | ((unsigned)s_comp[y & 0xFFu] << 24);
            }
            *reinterpret_cast<uint4 *>(out + p) = v;
        } else if (p < B1) {
            // a record boundary (or the end) inside the chunk: walk forward
            // from the step's record, one offset per record passed
            long long rr = r, ss = s, ee = e;
            for (int q = 0; q < 16; ++q) {
                const long long P = p + q;
                if (P >= B1) break;
                while (P >= ee && rr + 1 < n_seq) {
                    ++rr;
                    ss = ee;
                    ee = so[rr + 1];
                }
                const long long m = ss + ee - 1 - P;
                if (P >= ss && P < ee && m >= 0 && m < n) out[P] = s_comp[in[m]];
            }
        }
        // the next step's record (warp-uniform: s, e and p0 are the same in every lane)
        const long long nx = p0 + kRStep;
        if (nx < B1 && nx >= e) {
            r = dnatok::warp_find_le(so, n_seq, nx);
            s = so[r];
            e = so[r + 1];
        }
    }
}

}  // namespace

extern "C" {

dnatok_status dnatok_feed(const int32_t *ids_d, const int64_t *id_offsets_d, int64_t row_begin,
                          int64_t n_rows, int64_t token_len, int64_t id_pad, void *out_d,
                          int32_t out_bytes, dnatok_cuda_stream stream) {
    dnatok_status st = feed_args_ok(ids_d, id_offsets_d, row_begin, n_rows, token_len, id_pad,
                                    out_bytes);
    if (st != DNATOK_OK) return st;
    if (n_rows > 0 && token_len > 0 && !out_d) return DNATOK_ERR_ARG;
    if ((uintptr_t)out_d & (uintptr_t)(out_bytes - 1)) return DNATOK_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long long *offs = reinterpret_cast<const long long *>(id_offsets_d);
    cudaError_t e = out_bytes == 8
                        ? launch_feed<long long>(ids_d, offs, row_begin, n_rows, token_len, id_pad, out_d, s)
                        : launch_feed<int>(ids_d, offs, row_begin, n_rows, token_len, id_pad, out_d, s);
    return e == cudaSuccess ? DNATOK_OK : DNATOK_ERR_CUDA;
}

dnatok_status dnatok_microbatch_rows(int64_t emb_batch_cap, int64_t tokens_per_call,
                                     int64_t token_len, int64_t *rows) {
    if (!rows || emb_batch_cap < 1 || tokens_per_call < 0 || token_len < 1) return DNATOK_ERR_ARG;
    int64_t b = tokens_per_call / token_len;
    if (b < 1) b = 1;
    *rows = b < emb_batch_cap ? b : emb_batch_cap;
    return DNATOK_OK;
}

dnatok_status dnatok_feed_pipeline(const int32_t *ids_d, const int64_t *id_offsets_d,
                                   int64_t n_rows, int64_t token_len, int64_t id_pad,
                                   int32_t out_bytes, int64_t rows_per_batch, void *buf0_d,
                                   void *buf1_d, dnatok_cuda_stream feed_stream,
                                   dnatok_cuda_stream consumer_stream,
                                   dnatok_feed_consumer consumer, void *user) {
    dnatok_status st = feed_args_ok(ids_d, id_offsets_d, 0, n_rows, token_len, id_pad, out_bytes);
    if (st != DNATOK_OK) return st;
    if (!consumer || rows_per_batch < 1 || !buf0_d || !buf1_d) return DNATOK_ERR_ARG;
    cudaStream_t fs = reinterpret_cast<cudaStream_t>(feed_stream);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(consumer_stream);
    void *buf[2] = {buf0_d, buf1_d};
    cudaEvent_t ready[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr}, entry = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&entry, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming);
    }
    // the ids come from work ordered on consumer_stream (the caller's
    // stream): the feed stream starts after everything enqueued there so far
    if (e == cudaSuccess && fs != cs) {
        e = cudaEventRecord(entry, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(fs, entry, 0);
    }
    st = e == cudaSuccess ? DNATOK_OK : DNATOK_ERR_CUDA;
    const long long *offs = reinterpret_cast<const long long *>(id_offsets_d);
    long long i = 0;
    for (long long lo = 0; st == DNATOK_OK && lo < n_rows; lo += rows_per_batch, ++i) {
        const long long nb = (n_rows - lo < rows_per_batch) ? n_rows - lo : rows_per_batch;
        const int b = (int)(i & 1);
        if (i >= 2) e = cudaStreamWaitEvent(fs, freed[b], 0);  // its consumer is done
        if (e == cudaSuccess)
            e = out_bytes == 8 ? launch_feed<long long>(ids_d, offs, lo, nb, token_len, id_pad, buf[b], fs)
                               : launch_feed<int>(ids_d, offs, lo, nb, token_len, id_pad, buf[b], fs);
        if (e == cudaSuccess) e = cudaEventRecord(ready[b], fs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready[b], 0);
        if (e != cudaSuccess) {
            st = DNATOK_ERR_CUDA;
            break;
        }
        if (consumer(user, lo, nb, buf[b], consumer_stream) != 0) {
            st = DNATOK_ERR_STATE;
            break;
        }
        e = cudaEventRecord(freed[b], cs);
        if (e != cudaSuccess) st = DNATOK_ERR_CUDA;
    }
    for (int j = 0; j < 2; ++j) {
        if (ready[j]) cudaEventDestroy(ready[j]);
        if (freed[j]) cudaEventDestroy(freed[j]);
    }
    if (entry) cudaEventDestroy(entry);
    return st;
}

dnatok_status dnatok_reverse_complement(const uint8_t *bytes_d, int64_t n_bytes,
                                        const int64_t *seq_offsets_d, int64_t n_seq,
                                        uint8_t *out_d, dnatok_cuda_stream stream) {
    if (n_bytes < 0 || n_seq < 0 || !seq_offsets_d || ((uintptr_t)seq_offsets_d & 7u))
        return DNATOK_ERR_ARG;
    if (n_bytes == 0) return DNATOK_OK;
    if (!bytes_d || !out_d || n_seq == 0) return DNATOK_ERR_ARG;
    if ((const uint8_t *)out_d < bytes_d + n_bytes && bytes_d < (const uint8_t *)out_d + n_bytes)
        return DNATOK_ERR_ARG;  // overlapping buffers
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one resident wave of warps, each owning a 512-byte-aligned range
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, revcomp_kernel, kRThreads, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long warps = (long long)(sms > 0 ? sms : 1) * per_sm * (kRThreads / 32);
    long long per_warp = (n_bytes + warps - 1) / warps;
    per_warp = (per_warp + kRStep - 1) / kRStep * kRStep;
    const long long grid = ((n_bytes + per_warp - 1) / per_warp + kRThreads / 32 - 1) / (kRThreads / 32);
    const int vec = ((uintptr_t)out_d & 15u) == 0;
    revcomp_kernel<<<(unsigned)grid, kRThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        bytes_d, n_bytes, reinterpret_cast<const long long *>(seq_offsets_d), n_seq, out_d, vec,
        per_warp);
    return cudaGetLastError() == cudaSuccess ? DNATOK_OK : DNATOK_ERR_CUDA;
}

}  // extern "C"
