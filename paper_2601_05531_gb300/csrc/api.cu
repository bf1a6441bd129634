// api.cu -- the C ABI: handle life cycle, validation, one-shot encode.
#include <cstdio>
#include <cstring>
#include <set>
#include <utility>

#include "handle.h"
#include "tile_kernel.cuh"

using namespace dnatok;

namespace {
thread_local std::string g_create_error;

void default_lut(int32_t *lut) {
    for (int b = 0; b < 256; ++b) lut[b] = 4;  // N-class
    const char *bases = "ACGT";
    for (int i = 0; i < 4; ++i) {
        lut[(unsigned char)bases[i]] = i;
        lut[(unsigned char)bases[i] + 32] = i;
    }
    lut['\n'] = lut['\r'] = lut[' '] = lut['\t'] = -1;
}
}  // namespace

namespace dnatok {

dnatok_status fail(dnatok_handle *h, dnatok_status st, const std::string &msg) {
    if (h) h->last_error = msg;
    else g_create_error = msg;
    return st;
}

dnatok_status fail_cuda(dnatok_handle *h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(h, DNATOK_ERR_NOMEM, m);
    return fail(h, DNATOK_ERR_CUDA, m);
}

long long tiles_for(long long n_bytes, int head_pad, int tile) {
    return (head_pad + n_bytes + tile - 1) / tile;
}

dnatok_status ensure_workspace(dnatok_handle *h, long long n_bytes, long long n_bnd,
                               const LaunchShape &sh, cudaStream_t s) {
    const long long tiles = tiles_for(n_bytes, 15, sh.tile) + 1;
    if (tiles > h->desc_cap) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            return fail(h, DNATOK_ERR_STATE, "workspace must grow during stream capture; call dnatok_reserve first");
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaDeviceSynchronize");
        long long cap = tiles + tiles / 4 + 64;
        TileDesc *d = nullptr;
        e = cudaMalloc(&d, sizeof(TileDesc) * cap);
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMalloc(look-back descriptors)");
        e = cudaMemset(d, 0, sizeof(TileDesc) * cap);
        if (e != cudaSuccess) { cudaFree(d); return fail_cuda(h, e, "cudaMemset"); }
        int *r = nullptr;
        e = cudaMalloc(&r, sizeof(int) * (cap + 1));
        if (e != cudaSuccess) { cudaFree(d); return fail_cuda(h, e, "cudaMalloc(tile map)"); }
        cudaFree(h->d_desc);
        cudaFree(h->d_tile_rec);
        h->d_desc = d;
        h->d_tile_rec = r;
        h->desc_cap = cap;
        h->rec_cap = cap;
        e = cudaMemset(h->d_gate, 0, sizeof(unsigned));  // no old epoch left in the switch
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemset(gate)");
        h->epoch = 0;  // fresh zeroed descriptors: epoch 0 is never used
    }
    (void)n_bnd;
    return DNATOK_OK;
}

dnatok_status next_epoch(dnatok_handle *h, cudaStream_t s, unsigned *epoch) {
    h->epoch++;
    if ((h->epoch & ((1u << kEpochBits) - 1)) == 0) {  // epoch wrap: forget every old descriptor
        // The gate holds whole 32-bit epochs, so it needs clearing only when
        // those wrap; clearing it here could drop a gate that a direct path
        // raised for the general launch that takes this epoch.
        cudaError_t e = cudaMemsetAsync(h->d_desc, 0, sizeof(TileDesc) * h->desc_cap, s);
        if (e == cudaSuccess && h->epoch == 0) e = cudaMemsetAsync(h->d_gate, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemsetAsync(descriptors)");
        h->epoch++;
    }
    *epoch = h->epoch;
    return DNATOK_OK;
}

dnatok_status run_tile_encode(dnatok_handle *h, int mode, int k, int bsrc, const uint8_t *bytes,
                              long long n_bytes, const long long *seq_offsets, long long n_bnd,
                              void *out, long long out_cap, long long *offsets_out,
                              long long offsets_cap, long long *totals_out, const Carry *carry_in,
                              Carry *carry_out, int start_boundary, int end_boundary,
                              cudaStream_t s, unsigned gate_epoch) {
    const LaunchShape sh = h->shape;
    dnatok_status st = ensure_workspace(h, n_bytes, n_bnd, sh, s);
    if (st != DNATOK_OK) return st;
    TileParams p;
    std::memset(&p, 0, sizeof(p));
    p.bytes = bytes;
    p.n_bytes = n_bytes;
    p.seq_offsets = seq_offsets;
    p.n_bnd = n_bnd;
    p.out = out;
    p.out_cap = out_cap;
    p.offsets_out = offsets_out;
    p.offsets_cap = offsets_cap;
    p.totals_out = totals_out;
    p.desc = h->d_desc;
    p.tile_counter = h->d_counter;  // reset by the last CTA of every launch
    p.carry_in = carry_in;
    p.carry_out = carry_out;
    p.status = h->d_status;
    p.lut = h->d_lut;
    p.k = k;
    p.start_boundary = start_boundary;
    p.end_boundary = end_boundary;
    p.head_pad = (int)((uintptr_t)bytes & 15u);
    p.spin_limit = h->spin_limit;
    p.skip_chunk = h->skip_chunk;
    h->skip_chunk = -1;  // one launch only
    p.lut_keeps_bases = 1;
    for (const char *c = "ACGTacgt"; *c; ++c)
        if (h->lut_host[(unsigned char)*c] < 0) p.lut_keeps_bases = 0;
    cudaError_t e;
    h->direct_epoch = 0;
    if (n_bytes == 0) {
        e = launch_empty_chunk(p, bsrc == BSRC_LIST, s);
        if (e != cudaSuccess) return fail_cuda(h, e, "empty-chunk launch");
        return DNATOK_OK;
    }
    p.n_tiles = tiles_for(n_bytes, p.head_pad, sh.tile);
    p.n_chunks = (p.n_tiles + sh.chunk_tiles - 1) / sh.chunk_tiles;
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(s, &capst) == cudaSuccess &&
                           capst != cudaStreamCaptureStatusNone;
    if (gate_epoch != 0) {
        // behind a direct path of the caller's (launched before this call
        // on the same stream, never under capture): run only if it raised
        // the gate
        p.gate = h->d_gate;
        p.gate_epoch = gate_epoch;
    } else if (bsrc == BSRC_LIST && !carry_in && !carry_out && h->direct &&
               direct_eligible(mode, n_bnd - 1, h->lut_host)) {
        // RAW input: the direct path, with the general kernel behind it
        unsigned ep = 0;
        st = next_epoch(h, s, &ep);
        if (st != DNATOK_OK) return st;
        // under stream capture the epochs are baked into the graph: a replay
        // whose general kernel ran clears the switch and its descriptors at
        // its end (clear_gate), so the next replay starts clean
        const bool timed = h->ktime_on && mode == MODE_KMER && k >= 2 && !capturing;
        e = launch_direct(mode, bytes, n_bytes, seq_offsets, n_bnd - 1, out, offsets_out,
                          totals_out, h->d_gate, ep, k, h->d_lut, h->sm_count, h->dshape, s,
                          nullptr, 0x7fffffffffffffffll, timed ? h->ktime[0] : nullptr,
                          timed ? h->ktime[1] : nullptr);
        if (timed && e == cudaSuccess) h->ktime_valid = true;
        if (e != cudaSuccess) return fail_cuda(h, e, "direct kernel launch");
        p.gate = h->d_gate;
        p.gate_epoch = ep;
        h->direct_epoch = ep;
        if (capturing) p.clear_gate = h->d_gate;
    } else if (bsrc == BSRC_FASTA && fasta_direct_eligible(h, mode, k, bytes, n_bytes) &&
               (start_boundary ? !carry_in : carry_in != nullptr)) {
        // FASTA text (one-shot, or a chunk of a stream): compacted to sequence
        // bytes and record starts, then the direct path over them; the
        // general kernel behind it reads the text
        unsigned ep = 0;
        st = next_epoch(h, s, &ep);
        if (st != DNATOK_OK) return st;
        st = fasta_direct(h, bytes, n_bytes, out, out_cap, offsets_out, offsets_cap, totals_out,
                          carry_in, carry_out, start_boundary, end_boundary, ep, k, s);
        if (st != DNATOK_OK) return st;
        p.gate = h->d_gate;
        p.gate_epoch = ep;
        h->direct_epoch = ep;
        if (capturing) p.clear_gate = h->d_gate;
    }
    st = next_epoch(h, s, &p.epoch);
    if (st != DNATOK_OK) return st;
    {
        // Under stream capture the epoch is baked into the graph and every
        // replay reuses it, so the graph clears the descriptors it uses first.
        if (capturing && !p.gate) {
            e = cudaMemsetAsync(h->d_desc, 0, sizeof(TileDesc) * (size_t)p.n_chunks, s);
            if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemsetAsync(descriptors)");
        }
    }
    e = launch_tile_kernel(mode, bsrc, p, sh, s, h->sm_count);
    if (e != cudaSuccess) return fail_cuda(h, e, "tile kernel launch");
    return DNATOK_OK;
}

}  // namespace dnatok

// ======================================================================= ABI

extern "C" {

dnatok_status dnatok_create(dnatok_handle **out, dnatok_mode mode, int k,
                            const dnatok_tables *tables, dnatok_format fmt) {
    if (!out) return fail(nullptr, DNATOK_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (mode != DNATOK_CHAR && mode != DNATOK_KMER && mode != DNATOK_BPE &&
        mode != DNATOK_KMER_OVERLAP && mode != DNATOK_KMER_TABLE)
        return fail(nullptr, DNATOK_ERR_ARG, "unknown mode");
    if (fmt != DNATOK_RAW && fmt != DNATOK_FASTA)
        return fail(nullptr, DNATOK_ERR_ARG, "unknown format");
    if ((mode == DNATOK_KMER || mode == DNATOK_KMER_OVERLAP) && (k < 1 || k > DNATOK_MAX_K))
        return fail(nullptr, DNATOK_ERR_ARG, "k must be in [1, 15]");
    long long n_index = 0;
    if (mode == DNATOK_KMER_TABLE) {
        if (k < 1 || k > DNATOK_MAX_K_TABLE)
            return fail(nullptr, DNATOK_ERR_ARG, "k must be in [1, 10] for DNATOK_KMER_TABLE");
        if (!tables || !tables->kmer_lut || !tables->base_ids)
            return fail(nullptr, DNATOK_ERR_TABLE, "DNATOK_KMER_TABLE needs kmer_lut and base_ids");
        n_index = 1;
        for (int i = 0; i < k; ++i) n_index *= 5;
        for (long long i = 0; i < n_index; ++i)
            if (tables->kmer_lut[i] < -1)
                return fail(nullptr, DNATOK_ERR_TABLE, "kmer_lut ids must be >= -1");
        for (int d = 0; d < 5; ++d)
            if (tables->base_ids[d] < 0)
                return fail(nullptr, DNATOK_ERR_TABLE, "base_ids must be >= 0");
    }
    dnatok_handle *h = new (std::nothrow) dnatok_handle();
    if (!h) return fail(nullptr, DNATOK_ERR_NOMEM, "host allocation failed");
    h->mode = mode;
    h->k = (mode == DNATOK_KMER || mode == DNATOK_KMER_OVERLAP || mode == DNATOK_KMER_TABLE) ? k : 1;
    if (mode == DNATOK_KMER_TABLE) {
        h->klut_host.assign(tables->kmer_lut, tables->kmer_lut + n_index);
        for (int d = 0; d < 5; ++d) h->base_ids[d] = tables->base_ids[d];
    }
    if (mode == DNATOK_BPE && tables && tables->merges && tables->n_merges > 0)
        h->merges_host.assign(tables->merges, tables->merges + 2 * (size_t)tables->n_merges);
    h->fmt = fmt;
    if (mode == DNATOK_CHAR && tables && tables->ascii_lut256) {
        for (int b = 0; b < 256; ++b) {
            if (tables->ascii_lut256[b] < -1) {
                delete h;
                return fail(nullptr, DNATOK_ERR_TABLE, "LUT ids must be >= -1");
            }
            h->lut_host[b] = tables->ascii_lut256[b];
        }
    } else {
        default_lut(h->lut_host);
    }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_lut, sizeof(int) * 256);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_lut, h->lut_host, sizeof(int) * 256, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_counter, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_counter, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_gate, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(h->d_gate, 0, sizeof(unsigned));
    if (e == cudaSuccess && mode == DNATOK_KMER_TABLE) {
        e = cudaMalloc(&h->d_klut, sizeof(int32_t) * (size_t)n_index);
        if (e == cudaSuccess)
            e = cudaMemcpy(h->d_klut, h->klut_host.data(), sizeof(int32_t) * (size_t)n_index,
                           cudaMemcpyHostToDevice);
        // a u16 copy that fits shared memory (31 KB for k = 6), padded to 16 bytes
        bool small = k <= 6;
        for (long long i = 0; small && i < n_index; ++i) small = h->klut_host[i] < 0xFFFF;
        // 2-byte window entries for the direct path: ids below 0x8000, and a
        // window's base-5 index (5^k values) in 14 bits
        h->kent16 = k <= 6;
        for (long long i = 0; h->kent16 && i < n_index; ++i) h->kent16 = h->klut_host[i] < 0x8000;
        if (e == cudaSuccess && small) {
            std::vector<uint16_t> t16((size_t)((n_index + 7) / 8 * 8), 0xFFFF);
            for (long long i = 0; i < n_index; ++i)
                t16[i] = h->klut_host[i] < 0 ? (uint16_t)0xFFFF : (uint16_t)h->klut_host[i];
            e = cudaMalloc(&h->d_klut16, sizeof(uint16_t) * t16.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(h->d_klut16, t16.data(), sizeof(uint16_t) * t16.size(),
                               cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        std::string m = std::string("CUDA setup failed: ") + cudaGetErrorString(e);
        dnatok_destroy(h);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? DNATOK_ERR_NOMEM : DNATOK_ERR_CUDA, m);
    }
    if (mode == DNATOK_BPE) {
        if (!tables || (tables->n_merges > 0 && !tables->merges)) {
            dnatok_destroy(h);
            return fail(nullptr, DNATOK_ERR_TABLE, "BPE needs a merge table");
        }
        dnatok_status st = bpe_create(h, tables->merges, tables->n_merges);
        if (st != DNATOK_OK) {
            std::string m = h->last_error;
            dnatok_destroy(h);
            return fail(nullptr, st, m);
        }
    }
    *out = h;
    return DNATOK_OK;
}

void dnatok_destroy(dnatok_handle *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    stream_destroy(h);
    part_destroy(h);
    bpe_destroy(h);
    ovl_destroy(h);
    fasta_destroy(h);
    for (cudaEvent_t ev : h->ktime)
        if (ev) cudaEventDestroy(ev);
    dec_destroy(h);
    cudaFree(h->d_klut);
    cudaFree(h->d_klut16);
    cudaFree(h->d_lut);
    cudaFree(h->d_desc);
    cudaFree(h->d_tile_rec);
    cudaFree(h->d_counter);
    cudaFree(h->d_status);
    cudaFree(h->d_gate);
    cudaFree(h->d_stage_bytes);
    cudaFree(h->d_stage_offs);
    cudaFree(h->d_stage_out_offs);
    cudaFree(h->d_stage_totals);
    delete h;
}

dnatok_status dnatok_max_tokens(const dnatok_handle *h, int64_t n_bytes, int64_t n_seq,
                                int64_t *cap) {
    if (!h || !cap || n_bytes < 0 || n_seq < 0) return DNATOK_ERR_ARG;
    int64_t c = n_bytes;
    if (h->mode == DNATOK_KMER && h->fmt == DNATOK_RAW && h->k > 1) {
        const int64_t alt = (n_bytes + n_seq * (int64_t)(h->k - 1)) / h->k;
        if (alt < c) c = alt;
    }
    *cap = c;
    return DNATOK_OK;
}

dnatok_status dnatok_reserve(dnatok_handle *h, int64_t max_bytes, int64_t max_seq) {
    if (!h || max_bytes < 0 || max_seq < 0) return DNATOK_ERR_ARG;
    dnatok_status st = ensure_workspace(h, max_bytes, max_seq + 1, h->shape, 0);
    if (st != DNATOK_OK) return st;
    if (h->mode == DNATOK_BPE) return bpe_reserve(h, max_bytes);
    if (h->mode == DNATOK_KMER_OVERLAP || h->mode == DNATOK_KMER_TABLE)
        return ovl_reserve(h, max_bytes, h->fmt == DNATOK_RAW ? max_seq + 1 : max_bytes + 2, 0);
    if (h->fmt == DNATOK_FASTA && h->mode == DNATOK_KMER && h->k >= 2)
        return fasta_reserve(h, max_bytes, 1ll << 40, 0);  // the record starts at full size
    return DNATOK_OK;
}

dnatok_status dnatok_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                            const int64_t *seq_offsets_d, int64_t n_seq, int32_t *ids_out_d,
                            int64_t ids_capacity, int64_t *id_offsets_d,
                            int64_t offsets_capacity, int64_t *totals_d,
                            dnatok_cuda_stream stream) {
    if (!h) return DNATOK_ERR_ARG;
    if (n_bytes < 0 || (n_bytes > 0 && !bytes_d))
        return fail(h, DNATOK_ERR_ARG, "bad input bytes");
    if (!id_offsets_d) return fail(h, DNATOK_ERR_ARG, "id_offsets is NULL");
    if (((uintptr_t)id_offsets_d | (uintptr_t)seq_offsets_d | (uintptr_t)totals_d) & 7u)
        return fail(h, DNATOK_ERR_ARG, "int64 arrays must be 8-byte aligned");
    if ((uintptr_t)ids_out_d & 3u) return fail(h, DNATOK_ERR_ARG, "ids_out must be 4-byte aligned");
    if (h->fmt == DNATOK_RAW) {
        if (!seq_offsets_d || n_seq < 0) return fail(h, DNATOK_ERR_ARG, "RAW needs seq_offsets");
        if (n_seq >= INT32_MAX - 1) return fail(h, DNATOK_ERR_ARG, "too many sequences");
        if (offsets_capacity < n_seq + 1)
            return fail(h, DNATOK_ERR_CAPACITY, "id_offsets needs n_seq + 1 entries");
        if (n_seq == 0 && n_bytes != 0)
            return fail(h, DNATOK_ERR_ARG, "bytes without sequences");
    } else if (offsets_capacity < 1) {
        return fail(h, DNATOK_ERR_CAPACITY, "id_offsets needs at least one entry");
    }
    int64_t need = 0;
    dnatok_max_tokens(h, n_bytes, n_seq, &need);
    if (ids_capacity < need || (need > 0 && !ids_out_d))
        return fail(h, DNATOK_ERR_CAPACITY, "ids_out smaller than dnatok_max_tokens()");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (h->mode == DNATOK_BPE)
        return bpe_encode(h, bytes_d, n_bytes, seq_offsets_d, n_seq, ids_out_d, ids_capacity,
                          id_offsets_d, offsets_capacity, totals_d, s);
    if (h->mode == DNATOK_KMER_OVERLAP)
        return ovl_encode(h, bytes_d, n_bytes, seq_offsets_d, n_seq, ids_out_d, ids_capacity,
                          id_offsets_d, offsets_capacity, totals_d, s);
    if (h->mode == DNATOK_KMER_TABLE)
        return ktab_encode(h, bytes_d, n_bytes, seq_offsets_d, n_seq, ids_out_d, ids_capacity,
                           id_offsets_d, offsets_capacity, totals_d, s);
    const int mode = (h->mode == DNATOK_CHAR) ? MODE_CHAR : MODE_KMER;
    if (h->fmt == DNATOK_RAW)
        return run_tile_encode(h, mode, h->k, BSRC_LIST, bytes_d, n_bytes,
                               reinterpret_cast<const long long *>(seq_offsets_d), n_seq + 1,
                               ids_out_d, ids_capacity, reinterpret_cast<long long *>(id_offsets_d),
                               offsets_capacity, reinterpret_cast<long long *>(totals_d), nullptr,
                               nullptr, 0, 0, s);
    return run_tile_encode(h, mode, h->k, BSRC_FASTA, bytes_d, n_bytes, nullptr, 0, ids_out_d,
                           ids_capacity, reinterpret_cast<long long *>(id_offsets_d),
                           offsets_capacity, reinterpret_cast<long long *>(totals_d), nullptr,
                           nullptr, 1, 1, s);
}

static dnatok_status grow(dnatok_handle *h, void **buf, long long *cap, long long need,
                          size_t elem, const char *what) {
    if (need <= *cap) return DNATOK_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaDeviceSynchronize");
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    long long c = need + need / 8 + 64;
    e = cudaMalloc(buf, elem * c);
    if (e != cudaSuccess) return fail_cuda(h, e, what);
    *cap = c;
    return DNATOK_OK;
}

dnatok_status dnatok_encode_host(dnatok_handle *h, const uint8_t *host_bytes, int64_t n_bytes,
                                 const int64_t *host_seq_offsets, int64_t n_seq, int32_t *ids_out_d,
                                 int64_t ids_capacity, int64_t *id_offsets_host,
                                 int64_t offsets_capacity, int64_t *totals_host,
                                 dnatok_cuda_stream stream) {
    if (!h) return DNATOK_ERR_ARG;
    if (n_bytes < 0 || (n_bytes > 0 && !host_bytes)) return fail(h, DNATOK_ERR_ARG, "bad input bytes");
    if (h->fmt == DNATOK_RAW && (!host_seq_offsets || n_seq < 0))
        return fail(h, DNATOK_ERR_ARG, "RAW needs seq_offsets");
    if (!id_offsets_host || offsets_capacity < 1) return fail(h, DNATOK_ERR_ARG, "bad id_offsets");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    dnatok_status st = grow(h, (void **)&h->d_stage_bytes, &h->stage_bytes_cap, n_bytes, 1,
                            "cudaMalloc(staging bytes)");
    if (st != DNATOK_OK) return st;
    const long long n_off_in = (h->fmt == DNATOK_RAW) ? n_seq + 1 : 0;
    st = grow(h, (void **)&h->d_stage_offs, &h->stage_offs_cap, n_off_in, 8, "cudaMalloc(staging offsets)");
    if (st != DNATOK_OK) return st;
    st = grow(h, (void **)&h->d_stage_out_offs, &h->stage_out_offs_cap, offsets_capacity, 8,
              "cudaMalloc(staging id offsets)");
    if (st != DNATOK_OK) return st;
    if (!h->d_stage_totals) {
        cudaError_t e = cudaMalloc(&h->d_stage_totals, 2 * sizeof(long long));
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMalloc(totals)");
    }
    cudaError_t e = cudaSuccess;
    if (n_bytes > 0)
        e = cudaMemcpyAsync(h->d_stage_bytes, host_bytes, n_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_off_in > 0)
        e = cudaMemcpyAsync(h->d_stage_offs, host_seq_offsets, 8 * n_off_in, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemcpyAsync(H2D)");
    st = dnatok_encode(h, h->d_stage_bytes, n_bytes,
                       h->fmt == DNATOK_RAW ? reinterpret_cast<int64_t *>(h->d_stage_offs) : nullptr,
                       n_seq, ids_out_d, ids_capacity,
                       reinterpret_cast<int64_t *>(h->d_stage_out_offs), offsets_capacity,
                       reinterpret_cast<int64_t *>(h->d_stage_totals), stream);
    if (st != DNATOK_OK) return st;
    long long tot[2] = {0, 0};
    e = cudaMemcpyAsync(tot, h->d_stage_totals, sizeof(tot), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemcpyAsync(D2H totals)");
    const long long n_write = (tot[1] + 1 < offsets_capacity) ? tot[1] + 1 : offsets_capacity;
    e = cudaMemcpyAsync(id_offsets_host, h->d_stage_out_offs, 8 * n_write, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemcpyAsync(D2H offsets)");
    if (totals_host) {
        totals_host[0] = tot[0];
        totals_host[1] = tot[1];
    }
    return dnatok_sync(h, stream);
}

dnatok_status dnatok_sync(dnatok_handle *h, dnatok_cuda_stream stream) {
    if (!h) return DNATOK_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaStreamSynchronize");
    int st = 0;
    e = cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(h, e, "status read");
    if (st == DEV_OK) return DNATOK_OK;
    const int zero = 0;
    cudaMemcpy(h->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    // a launch that stopped early may have left its tile counters set
    cudaMemset(h->d_counter, 0, 2 * sizeof(unsigned long long));
    if (st == DEV_TIMEOUT) return fail(h, DNATOK_ERR_TIMEOUT, "a bounded device wait ran out");
    if (st == DEV_CAPACITY)
        return fail(h, DNATOK_ERR_CAPACITY, "id_offsets has no room for every record found");
    if (st == DEV_BAD_OFFSETS)
        return fail(h, DNATOK_ERR_DEVICE_DATA,
                    "seq_offsets malformed (must be non-decreasing, [0]=0, [n_seq]=n_bytes)");
    return fail(h, DNATOK_ERR_CUDA, "device reported error " + std::to_string(st));
}

dnatok_status dnatok_last_error(const dnatok_handle *h, char *buf, size_t len) {
    if (!buf || len == 0) return DNATOK_ERR_ARG;
    const std::string &m = h ? h->last_error : g_create_error;
    std::snprintf(buf, len, "%s", m.c_str());
    return DNATOK_OK;
}

dnatok_status dnatok_get_launch(const dnatok_handle *h, dnatok_launch_cfg *cfg) {
    if (!h || !cfg) return DNATOK_ERR_ARG;
    cfg->tile_bytes = h->shape.tile;
    cfg->threads = h->shape.threads;
    cfg->ctas_per_sm = h->shape.ctas_per_sm;
    cfg->chunk_tiles = h->shape.chunk_tiles;
    return DNATOK_OK;
}

dnatok_status dnatok_set_direct_launch(dnatok_handle *h, int32_t slots_per_step, int32_t ring_steps,
                                       int32_t ctas_per_sm) {
    if (!h) return DNATOK_ERR_ARG;
    const DirectShape sh{slots_per_step, ring_steps, ctas_per_sm};
    if (!direct_shape_supported(sh)) return fail(h, DNATOK_ERR_ARG, "unsupported direct shape");
    h->dshape = sh;
    return DNATOK_OK;
}

dnatok_status dnatok_get_direct_launch(const dnatok_handle *h, int32_t *out3) {
    if (!h || !out3) return DNATOK_ERR_ARG;
    out3[0] = h->dshape.slots;
    out3[1] = h->dshape.ring;
    out3[2] = h->dshape.ctas_per_sm;
    return DNATOK_OK;
}

dnatok_status dnatok_set_direct(dnatok_handle *h, int32_t enable) {
    if (!h || (enable != 0 && enable != 1)) return DNATOK_ERR_ARG;
    h->direct = enable != 0;
    return DNATOK_OK;
}

dnatok_status dnatok_direct_ran(dnatok_handle *h, dnatok_cuda_stream stream, int32_t *out) {
    if (!h || !out) return DNATOK_ERR_ARG;
    *out = -1;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaStreamSynchronize");
    if (h->direct_epoch == 0) return DNATOK_OK;
    unsigned g = 0;
    e = cudaMemcpy(&g, h->d_gate, sizeof(g), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemcpy(gate)");
    *out = (g == h->direct_epoch) ? 0 : 1;
    return DNATOK_OK;
}

dnatok_status dnatok_set_kernel_timing(dnatok_handle *h, int32_t enable) {
    if (!h) return DNATOK_ERR_ARG;
    if (enable && !h->ktime[0]) {
        cudaError_t e = cudaEventCreate(&h->ktime[0]);
        if (e == cudaSuccess) e = cudaEventCreate(&h->ktime[1]);
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaEventCreate");
    }
    h->ktime_on = enable != 0;
    h->ktime_valid = false;
    return DNATOK_OK;
}

dnatok_status dnatok_kernel_time_ms(dnatok_handle *h, dnatok_cuda_stream stream, float *ms) {
    if (!h || !ms) return DNATOK_ERR_ARG;
    *ms = -1.0f;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaStreamSynchronize");
    if (!h->ktime_valid) return DNATOK_OK;
    e = cudaEventElapsedTime(ms, h->ktime[0], h->ktime[1]);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaEventElapsedTime");
    return DNATOK_OK;
}

dnatok_status dnatok_set_wait_limit(dnatok_handle *h, int64_t polls) {
    if (!h || polls < 0) return DNATOK_ERR_ARG;
    h->spin_limit = polls == 0 ? kSpinLimit : polls;
    return DNATOK_OK;
}

dnatok_status dnatok_inject_lookback_stall(dnatok_handle *h, int64_t chunk) {
    if (!h || chunk < -1) return DNATOK_ERR_ARG;
    h->skip_chunk = chunk;
    return DNATOK_OK;
}

dnatok_status dnatok_set_bpe_launch(dnatok_handle *h, int32_t seg_symbols, int32_t halo) {
    if (!h) return DNATOK_ERR_ARG;
    return bpe_set_launch(h, seg_symbols, halo);
}

dnatok_status dnatok_get_bpe_launch(const dnatok_handle *h, int32_t *seg_symbols, int32_t *halo) {
    if (!h || !seg_symbols || !halo) return DNATOK_ERR_ARG;
    return bpe_get_launch(h, seg_symbols, halo);
}

dnatok_status dnatok_bpe_stats(dnatok_handle *h, int64_t *stats3, dnatok_cuda_stream stream) {
    if (!h || !stats3) return DNATOK_ERR_ARG;
    long long v[3];
    const dnatok_status st = bpe_stats(h, v, reinterpret_cast<cudaStream_t>(stream));
    if (st != DNATOK_OK) return st;
    for (int i = 0; i < 3; ++i) stats3[i] = v[i];
    return DNATOK_OK;
}

dnatok_status dnatok_set_launch(dnatok_handle *h, const dnatok_launch_cfg *cfg) {
    if (!h || !cfg) return DNATOK_ERR_ARG;
    LaunchShape sh{cfg->tile_bytes, cfg->threads, cfg->ctas_per_sm, cfg->chunk_tiles};
    if (!tile_shape_supported(sh) || sh.ctas_per_sm < 1 || sh.ctas_per_sm > 8)
        return fail(h, DNATOK_ERR_ARG, "unsupported launch shape");
    h->shape = sh;
    return DNATOK_OK;
}

}  // extern "C"
