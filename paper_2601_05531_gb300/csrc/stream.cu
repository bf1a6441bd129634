// stream.cu -- host-streamed encode: pinned staging, a ring of device slots,
// a copy stream and a compute stream (Sec. 2.2 "Encoding paths": pinned
// staging of raw bytes, and the pipelined path's overlap of the transfer of
// one batch with the work on the previous one).
//
// Each submitted piece is cut into chunks.  Chunk i goes to device slot
// i % n_slots: its H2D copy waits (on the copy stream) for the kernel that
// last read the slot; its kernel waits (on the compute stream) for the copy.
// FASTA k-mer chunks of 64 KiB and more take the compacted path (fasta.cu),
// the others the general kernel; both read and write the same carry.
// Kernels run in stream order and pass the scan state through a two-entry
// device carry (chunk i reads carry[i & 1] and writes carry[(i + 1) & 1]), so
// the ids and offsets land at their global positions exactly as one
// dnatok_encode of the concatenated stream would put them.
#include <cstring>
#include <vector>

#include "handle.h"
#include "tile_kernel.cuh"

using namespace dnatok;

namespace {
constexpr int kProgSlots = 1024;  // request results remembered for poll

struct Progress {
    long long totals[2];  // {ids, records} through the request
    int status;           // device status word after the request
    int pad;
};
}  // namespace

struct StreamState {
    int32_t *ids = nullptr;
    long long ids_cap = 0;
    long long *offs = nullptr;
    long long offs_cap = 0;

    long long chunk = 64ll << 20;
    int n_slots = 3;
    int overlap = 1;
    cudaStream_t copy_s = nullptr, comp_s = nullptr;
    std::vector<uint8_t *> d_slot;
    std::vector<uint8_t *> h_slot;  // page-locked ring, allocated on first pageable submit
    std::vector<cudaEvent_t> copied;    // H2D into slot done (host slot reusable)
    std::vector<cudaEvent_t> consumed;  // kernel reading slot done (device slot reusable)
    long long slot_seq = 0;

    Carry *d_carry = nullptr;  // two entries, ping-pong
    int carry_cur = 0;
    bool any_launch = false;
    long long *d_tot = nullptr;

    Progress *h_prog = nullptr;  // page-locked, kProgSlots entries
    cudaEvent_t prog_ev[kProgSlots] = {};
    unsigned long long prog_req[kProgSlots] = {};
    long long prog_bytes[kProgSlots] = {};
    unsigned long long next_req = 0;

    long long bytes_in = 0;
    bool started = false;  // a start boundary has been placed
    bool ended = false;
};

namespace dnatok {

void stream_destroy(dnatok_handle *h) {
    StreamState *st = h->stream;
    if (!st) return;
    if (st->comp_s) cudaStreamSynchronize(st->comp_s);
    if (st->copy_s) cudaStreamSynchronize(st->copy_s);
    for (auto p : st->d_slot) cudaFree(p);
    for (auto p : st->h_slot) cudaFreeHost(p);
    for (auto e : st->copied) cudaEventDestroy(e);
    for (auto e : st->consumed) cudaEventDestroy(e);
    for (auto e : st->prog_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(st->d_carry);
    cudaFree(st->d_tot);
    if (st->h_prog) cudaFreeHost(st->h_prog);
    if (st->copy_s) cudaStreamDestroy(st->copy_s);
    if (st->comp_s) cudaStreamDestroy(st->comp_s);
    delete st;
    h->stream = nullptr;
}

}  // namespace dnatok

namespace {

dnatok_status stream_fail_cuda(dnatok_handle *h, cudaError_t e, const char *what) {
    return fail_cuda(h, e, what);
}

// One chunk (possibly empty) through the pipeline.
dnatok_status run_chunk(dnatok_handle *h, StreamState *st, const uint8_t *src, long long n,
                        bool pinned, int sb, int eb) {
    const int mode = (h->mode == DNATOK_CHAR) ? MODE_CHAR : MODE_KMER;
    const Carry *cin = st->any_launch ? st->d_carry + st->carry_cur : nullptr;
    Carry *cout = st->d_carry + (st->carry_cur ^ 1);
    if (n == 0) {
        // only boundaries: counted through the list-source path of the
        // zero-byte kernel (it reads no offsets, only their number)
        const long long nb = sb + eb;
        if (nb == 0) return DNATOK_OK;
        dnatok_status r = run_tile_encode(h, mode, h->k, BSRC_LIST, nullptr, 0, nullptr, nb,
                                          st->ids, st->ids_cap, st->offs, st->offs_cap, st->d_tot,
                                          cin, cout, 0, 0, st->comp_s);
        if (r != DNATOK_OK) return r;
        st->carry_cur ^= 1;
        st->any_launch = true;
        return DNATOK_OK;
    }
    const int slot = (int)(st->slot_seq++ % st->n_slots);
    cudaError_t e;
    if (!pinned) {
        // the page-locked slot is free once its previous H2D copy finished
        e = cudaEventSynchronize(st->copied[slot]);
        if (e != cudaSuccess) return stream_fail_cuda(h, e, "cudaEventSynchronize(ring slot)");
        std::memcpy(st->h_slot[slot], src, (size_t)n);
        src = st->h_slot[slot];
    }
    cudaStream_t cs = st->overlap ? st->copy_s : st->comp_s;
    e = cudaStreamWaitEvent(cs, st->consumed[slot], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st->d_slot[slot], src, (size_t)n, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(st->copied[slot], cs);
    if (e == cudaSuccess && st->overlap) e = cudaStreamWaitEvent(st->comp_s, st->copied[slot], 0);
    if (e != cudaSuccess) return stream_fail_cuda(h, e, "H2D chunk copy");
    const int bsrc = (h->fmt == DNATOK_FASTA) ? BSRC_FASTA : BSRC_FLAGS;
    dnatok_status r = run_tile_encode(h, mode, h->k, bsrc, st->d_slot[slot], n, nullptr, 0,
                                      st->ids, st->ids_cap, st->offs, st->offs_cap, st->d_tot,
                                      cin, cout, sb, eb, st->comp_s);
    if (r != DNATOK_OK) return r;
    st->carry_cur ^= 1;
    st->any_launch = true;
    e = cudaEventRecord(st->consumed[slot], st->comp_s);
    if (e != cudaSuccess) return stream_fail_cuda(h, e, "cudaEventRecord");
    return DNATOK_OK;
}

dnatok_status read_progress(dnatok_handle *h, StreamState *st, int r, dnatok_stream_result *out) {
    const Progress &pg = st->h_prog[r];
    if (pg.status != DEV_OK) {
        if (pg.status == DEV_TIMEOUT) return fail(h, DNATOK_ERR_TIMEOUT, "a bounded device wait ran out");
        return fail(h, DNATOK_ERR_CUDA, "device reported error " + std::to_string(pg.status));
    }
    if (out) {
        out->n_ids = pg.totals[0];
        out->n_records = pg.totals[1];
        out->bytes_in = st->prog_bytes[r];
    }
    if (pg.totals[0] > st->ids_cap)
        return fail(h, DNATOK_ERR_CAPACITY,
                    "ids_out too small: the stream has " + std::to_string(pg.totals[0]) + " ids");
    return DNATOK_OK;
}

}  // namespace

extern "C" {

dnatok_status dnatok_stream_open(dnatok_handle *h, const dnatok_stream_cfg *cfg,
                                 int32_t *ids_out_d, int64_t ids_capacity, int64_t *id_offsets_d,
                                 int64_t offsets_capacity) {
    if (!h) return DNATOK_ERR_ARG;
    if (h->stream) return fail(h, DNATOK_ERR_STATE, "a stream is already open on this handle");
    if (h->mode == DNATOK_BPE || h->mode == DNATOK_KMER_OVERLAP || h->mode == DNATOK_KMER_TABLE)
        return fail(h, DNATOK_ERR_STATE, "streams take CHAR or KMER handles");
    if (ids_capacity < 0 || (ids_capacity > 0 && !ids_out_d) || offsets_capacity < 0 ||
        (offsets_capacity > 0 && !id_offsets_d))
        return fail(h, DNATOK_ERR_ARG, "bad output arrays");
    long long chunk = 64ll << 20;
    int slots = 3, overlap = 1;
    if (cfg) {
        if (cfg->chunk_bytes < 0 || cfg->n_slots < 0 || cfg->n_slots == 1 || cfg->n_slots > 8 ||
            (cfg->overlap != 0 && cfg->overlap != 1))
            return fail(h, DNATOK_ERR_ARG, "bad stream configuration");
        if (cfg->chunk_bytes > 0) chunk = cfg->chunk_bytes;
        if (cfg->n_slots > 0) slots = cfg->n_slots;
        overlap = cfg->overlap;
    }
    StreamState *st = new (std::nothrow) StreamState();
    if (!st) return fail(h, DNATOK_ERR_NOMEM, "host allocation failed");
    h->stream = st;
    st->ids = ids_out_d;
    st->ids_cap = ids_capacity;
    st->offs = reinterpret_cast<long long *>(id_offsets_d);
    st->offs_cap = offsets_capacity;
    st->chunk = chunk;
    st->n_slots = slots;
    st->overlap = overlap;
    dnatok_status r = ensure_workspace(h, chunk, 0, h->shape, 0);
    if (r == DNATOK_OK && h->fmt == DNATOK_FASTA && h->mode == DNATOK_KMER && h->k >= 2)
        r = fasta_reserve(h, chunk, 1ll << 40, 0);  // the compacted path's workspace, up front
    if (r != DNATOK_OK) {
        stream_destroy(h);
        return r;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&st->comp_s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st->copy_s, cudaStreamNonBlocking);
    for (int i = 0; i < slots && e == cudaSuccess; ++i) {
        uint8_t *d = nullptr;
        e = cudaMalloc(&d, (size_t)chunk);
        if (e != cudaSuccess) break;
        st->d_slot.push_back(d);
        cudaEvent_t a = nullptr, b = nullptr;
        e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming);
        if (a) st->copied.push_back(a);
        if (b) st->consumed.push_back(b);
    }
    if (e == cudaSuccess) e = cudaMalloc(&st->d_carry, 2 * sizeof(Carry));
    if (e == cudaSuccess) e = cudaMalloc(&st->d_tot, 2 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(st->d_tot, 0, 2 * sizeof(long long));
    if (e == cudaSuccess) e = cudaHostAlloc(&st->h_prog, sizeof(Progress) * kProgSlots, cudaHostAllocDefault);
    for (int i = 0; i < kProgSlots && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&st->prog_ev[i], cudaEventDisableTiming);
        st->prog_req[i] = ~0ull;
    }
    if (e != cudaSuccess) {
        r = fail_cuda(h, e, "stream set-up");
        stream_destroy(h);
        return r;
    }
    std::memset(st->h_prog, 0, sizeof(Progress) * kProgSlots);
    return DNATOK_OK;
}

dnatok_status dnatok_stream_submit(dnatok_handle *h, const uint8_t *host_bytes, int64_t n,
                                   int flags, uint64_t *req_id) {
    if (!h) return DNATOK_ERR_ARG;
    StreamState *st = h->stream;
    if (!st) return fail(h, DNATOK_ERR_STATE, "no stream is open");
    if (st->ended) return fail(h, DNATOK_ERR_STATE, "the stream has ended");
    if (n < 0 || (n > 0 && !host_bytes) || !req_id ||
        (flags & ~(DNATOK_END_OF_STREAM | DNATOK_NEW_RECORD | DNATOK_HOST_PINNED)))
        return fail(h, DNATOK_ERR_ARG, "bad submit arguments");
    const bool pinned = (flags & DNATOK_HOST_PINNED) != 0;
    const bool end = (flags & DNATOK_END_OF_STREAM) != 0;
    if (!pinned && n > 0 && st->h_slot.empty()) {
        for (int i = 0; i < st->n_slots; ++i) {
            uint8_t *p = nullptr;
            cudaError_t e = cudaHostAlloc(&p, (size_t)st->chunk, cudaHostAllocDefault);
            if (e != cudaSuccess) return fail_cuda(h, e, "cudaHostAlloc(ring)");
            st->h_slot.push_back(p);
        }
    }
    const bool raw = (h->fmt == DNATOK_RAW);
    // RAW: the first piece and every NEW_RECORD piece start a record.
    // FASTA: the stream's first byte starts one (the kernel merges it with a
    // header that begins there), so it waits for the first non-empty chunk.
    int sb = 0;
    if (raw) sb = (!st->started || (flags & DNATOK_NEW_RECORD)) ? 1 : 0;
    else sb = (!st->started && n > 0) ? 1 : 0;
    if (sb) st->started = true;
    long long done = 0;
    do {
        const long long len = (n - done < st->chunk) ? n - done : st->chunk;
        const bool last = (done + len == n);
        dnatok_status r = run_chunk(h, st, host_bytes + done, len, pinned, sb, (end && last) ? 1 : 0);
        if (r != DNATOK_OK) return r;
        sb = 0;
        done += len;
    } while (done < n);
    st->bytes_in += n;
    if (end) st->ended = true;

    const unsigned long long id = st->next_req++;
    const int slot = (int)(id % kProgSlots);
    cudaError_t e = cudaSuccess;
    if (st->prog_req[slot] != ~0ull) e = cudaEventSynchronize(st->prog_ev[slot]);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st->h_prog[slot].totals, st->d_tot, 2 * sizeof(long long),
                            cudaMemcpyDeviceToHost, st->comp_s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&st->h_prog[slot].status, h->d_status, sizeof(int),
                            cudaMemcpyDeviceToHost, st->comp_s);
    if (e == cudaSuccess) e = cudaEventRecord(st->prog_ev[slot], st->comp_s);
    if (e != cudaSuccess) return fail_cuda(h, e, "request completion record");
    st->prog_req[slot] = id;
    st->prog_bytes[slot] = st->bytes_in;
    *req_id = id;
    return DNATOK_OK;
}

dnatok_status dnatok_stream_poll(dnatok_handle *h, uint64_t req_id, dnatok_stream_result *out) {
    if (!h) return DNATOK_ERR_ARG;
    StreamState *st = h->stream;
    if (!st) return fail(h, DNATOK_ERR_STATE, "no stream is open");
    const int slot = (int)(req_id % kProgSlots);
    if (req_id >= st->next_req || st->prog_req[slot] != req_id)
        return fail(h, DNATOK_ERR_UNKNOWN_REQ, "unknown or expired request id");
    cudaError_t e = cudaEventQuery(st->prog_ev[slot]);
    if (e == cudaErrorNotReady) return DNATOK_PENDING;
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaEventQuery");
    return read_progress(h, st, slot, out);
}

dnatok_status dnatok_stream_wait(dnatok_handle *h, uint64_t req_id, dnatok_stream_result *out) {
    if (!h) return DNATOK_ERR_ARG;
    StreamState *st = h->stream;
    if (!st) return fail(h, DNATOK_ERR_STATE, "no stream is open");
    const int slot = (int)(req_id % kProgSlots);
    if (req_id >= st->next_req || st->prog_req[slot] != req_id)
        return fail(h, DNATOK_ERR_UNKNOWN_REQ, "unknown or expired request id");
    cudaError_t e = cudaEventSynchronize(st->prog_ev[slot]);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaEventSynchronize");
    return read_progress(h, st, slot, out);
}

dnatok_status dnatok_stream_close(dnatok_handle *h) {
    if (!h) return DNATOK_ERR_ARG;
    StreamState *st = h->stream;
    if (!st) return fail(h, DNATOK_ERR_STATE, "no stream is open");
    cudaError_t e = cudaStreamSynchronize(st->comp_s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->copy_s);
    stream_destroy(h);
    if (e != cudaSuccess) return fail_cuda(h, e, "stream close");
    return dnatok_sync(h, 0);
}

}  // extern "C"
