// part.cu -- one long stream split into parts that separate processes (one
// per GPU) encode, the only exchange being a small summary per part.
//
// A part is a contiguous byte range of the stream.  What its encode needs
// from the bytes before it is the scan element at its start (records seen,
// tokens completed, kept symbols of the open record and its last k - 1
// codes: the Agg of the tile kernel's look-back) and, for FASTA, the line
// state there.  Each rank
//   1. computes its part's line-state map (three states to three: it
//      depends only on the part's first byte, its last newline and the byte
//      after that), and the ranks exchange the maps, so every rank knows the
//      line state at its start;
//   2. finds its part's own scan element (rank 0 encodes from the stream
//      start, which is its real encode), and the ranks exchange those;
//   3. combines the elements of the parts before it into its start element
//      and encodes its part from there: its ids land at the start of its own
//      buffer, its record offsets are global token positions.
// The encode of a part is the chunk encode of the host-streamed path
// (dnatok_stream_*), so a part's outputs equal the same slice of one encode
// of the whole stream.
#include <cstring>

#include "handle.h"
#include "tile_kernel.cuh"

using namespace dnatok;

namespace {

constexpr int kLnThreads = 256;

// 1 + the position of the last '\n' in bytes[0, n) (0: none), by atomicMax
// into *out (zeroed before).  16-byte loads over the aligned span around the
// bytes (they stay inside its 16-byte granules); a vector without a newline
// costs one SWAR test.
__global__ void __launch_bounds__(kLnThreads) last_newline_kernel(const uint8_t *bytes, long long n,
                                                                 unsigned long long *out) {
    const int head = (int)((uintptr_t)bytes & 15u);
    const uint4 *v = reinterpret_cast<const uint4 *>(bytes - head);
    const long long n_vec = (head + n + 15) / 16;
    unsigned long long best = 0;
    for (long long i = blockIdx.x * (long long)kLnThreads + threadIdx.x; i < n_vec;
         i += (long long)gridDim.x * kLnThreads) {
        const uint4 w = __ldg(v + i);
        const unsigned x[4] = {w.x ^ 0x0A0A0A0Au, w.y ^ 0x0A0A0A0Au, w.z ^ 0x0A0A0A0Au,
                               w.w ^ 0x0A0A0A0Au};
        bool any = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) any |= ((x[j] - 0x01010101u) & ~x[j] & 0x80808080u) != 0u;
        if (!any) continue;
        for (int j = 15; j >= 0; --j) {
            const long long pos = 16 * i + j - head;
            if (pos < 0 || pos >= n) continue;
            if (((x[j >> 2] >> (8 * (j & 3))) & 0xFFu) == 0u) {  // the byte was '\n'
                const unsigned long long c = (unsigned long long)pos + 1ull;
                if (c > best) best = c;
                break;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
        if (y > best) best = y;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

// The part's line-state map (hmap form: the end state of each start state,
// two bits each) from its first byte, its last newline and the byte after.
__global__ void line_map_kernel(const uint8_t *bytes, long long n, const unsigned long long *last_nl,
                                int *map) {
    if (n == 0) {
        *map = (int)kHmapIdentity;
        return;
    }
    const unsigned long long c = *last_nl;  // 1 + position, 0: none
    if (c == 0) {
        // no newline: a line start takes its state from the first byte,
        // inside a line the state stays
        const unsigned first = bytes[0] == '>' ? HS_HD : HS_SQ;
        *map = (int)(first | (HS_HD << 2) | (HS_SQ << 4));
        return;
    }
    unsigned end = HS_LS;  // the part ends with its newline
    if ((long long)c < n) end = bytes[c] == '>' ? HS_HD : HS_SQ;
    *map = (int)hmap_const(end);
}

// The host side of the look-back's scan element combine (the same rules as
// agg_combine, with plain divisions).
Agg host_combine(const Agg &A, const Agg &B, int k) {
    auto div = [k](long long x) { return k == 1 ? x : x / k; };
    Agg r;
    r.nb = A.nb + B.nb;
    if (A.nb == 0) {
        r.h = A.h + B.h;
        r.d = B.d;
        r.t = B.t;
    } else if (B.nb == 0) {
        r.h = A.h;
        r.d = A.d - div(A.t) + div(A.t + B.h);
        r.t = A.t + B.h;
    } else {
        r.h = A.h;
        r.d = A.d - div(A.t) + div(A.t + B.h + k - 1) + B.d;
        r.t = B.t;
    }
    r.codes = (B.nb > 0) ? B.codes : codes_concat(A.codes, B.codes, k);
    return r;
}

Carry to_carry(const dnatok_part_state &s) {
    Carry c;
    c.a.nb = s.nb;
    c.a.h = s.h;
    c.a.d = s.d;
    c.a.t = s.t;
    c.a.codes = s.codes;
    c.hstate = s.line_state;
    c.pad = 0;
    return c;
}

dnatok_part_state from_carry(const Carry &c) {
    dnatok_part_state s;
    s.nb = c.a.nb;
    s.h = c.a.h;
    s.d = c.a.d;
    s.t = c.a.t;
    s.codes = c.a.codes;
    s.line_state = c.hstate;
    s.pad = 0;
    return s;
}

dnatok_status part_scratch(dnatok_handle *h) {
    if (h->d_part) return DNATOK_OK;
    // [0, 2) carries in and out, then the newline position, the map, totals
    const size_t bytes = 2 * sizeof(Carry) + 64;
    cudaError_t e = cudaMalloc(&h->d_part, bytes);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMalloc(part workspace)");
    return DNATOK_OK;
}

Carry *part_carry(dnatok_handle *h) { return reinterpret_cast<Carry *>(h->d_part); }
unsigned long long *part_nl(dnatok_handle *h) {
    return reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(h->d_part) + 2 * sizeof(Carry));
}
int *part_map(dnatok_handle *h) { return reinterpret_cast<int *>(part_nl(h) + 1); }
long long *part_tot(dnatok_handle *h) { return reinterpret_cast<long long *>(part_nl(h) + 2); }

}  // namespace

namespace dnatok {
void part_destroy(dnatok_handle *h) {
    cudaFree(h->d_part);
    h->d_part = nullptr;
}
}  // namespace dnatok

extern "C" {

dnatok_status dnatok_part_line_map(dnatok_handle *h, const uint8_t *bytes_d, int64_t n,
                                   int32_t *map_out, dnatok_cuda_stream stream) {
    if (!h || !map_out || n < 0 || (n > 0 && !bytes_d)) return DNATOK_ERR_ARG;
    if (h->fmt != DNATOK_FASTA) {
        *map_out = (int32_t)kHmapIdentity;  // RAW: no line state
        return DNATOK_OK;
    }
    dnatok_status st = part_scratch(h);
    if (st != DNATOK_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(part_nl(h), 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemsetAsync");
    if (n > 0) {
        long long grid = ((((uintptr_t)bytes_d & 15u) + n + 15) / 16 + kLnThreads - 1) / kLnThreads;
        if (grid > (long long)h->sm_count * 8) grid = (long long)h->sm_count * 8;
        if (grid < 1) grid = 1;
        last_newline_kernel<<<(unsigned)grid, kLnThreads, 0, s>>>(bytes_d, n, part_nl(h));
    }
    line_map_kernel<<<1, 1, 0, s>>>(bytes_d, n, part_nl(h), part_map(h));
    int m = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&m, part_map(h), sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e, "line map");
    *map_out = m;
    return DNATOK_OK;
}

// One run of the chunk encode over the part from the device carry in slot 0
// (or from the stream start), ids and offsets placed from the stream-wide
// positions d0 and nb0; the carry out is copied to *c_out.
static dnatok_status part_run(dnatok_handle *h, int mode, int k, const uint8_t *bytes_d, long long n,
                              bool from_carry, long long d0, long long nb0, int eb,
                              int32_t *ids_out_d, long long ids_capacity, int64_t *id_offsets_d,
                              long long offsets_capacity, Carry *c_out, cudaStream_t s) {
    const Carry *cin = from_carry ? part_carry(h) : nullptr;
    Carry *cout = part_carry(h) + 1;
    // ids and offsets are placed at their stream-wide positions: shifted
    // bases put this part's first id and first record at the start of the
    // caller's arrays (nothing is written below them)
    int32_t *out = ids_out_d - d0;
    long long *offs = reinterpret_cast<long long *>(id_offsets_d) - nb0;
    const int sb = from_carry ? 0 : 1;
    dnatok_status st;
    if (n == 0) {
        // boundaries only; a FASTA stream with no bytes at all has no record
        // (its start is not one), as in a one-shot encode of no text
        const long long nb = (h->fmt == DNATOK_FASTA && !from_carry) ? eb : sb + eb;
        st = run_tile_encode(h, mode, k, BSRC_LIST, nullptr, 0, nullptr, nb, out,
                             ids_capacity + d0, offs, offsets_capacity + nb0, part_tot(h), cin, cout,
                             0, 0, s);
    } else {
        const int bsrc = (h->fmt == DNATOK_FASTA) ? BSRC_FASTA : BSRC_FLAGS;
        st = run_tile_encode(h, mode, k, bsrc, bytes_d, n, nullptr, 0, out, ids_capacity + d0, offs,
                             offsets_capacity + nb0, part_tot(h), cin, cout, sb, eb, s);
    }
    if (st != DNATOK_OK) return st;
    cudaError_t e = cudaMemcpyAsync(c_out, cout, sizeof(Carry), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemcpyAsync(part state)");
    return dnatok_sync(h, reinterpret_cast<dnatok_cuda_stream>(s));
}

dnatok_status dnatok_part_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n,
                                 const dnatok_part_state *before, int32_t last, int32_t *ids_out_d,
                                 int64_t ids_capacity, int64_t *id_offsets_d,
                                 int64_t offsets_capacity, dnatok_part_state *after,
                                 dnatok_cuda_stream stream) {
    if (!h || !after || n < 0 || (n > 0 && !bytes_d)) return DNATOK_ERR_ARG;
    if (h->mode != DNATOK_CHAR && h->mode != DNATOK_KMER)
        return fail(h, DNATOK_ERR_STATE, "parts of a stream: single-nucleotide and k-mer handles only");
    if (h->stream) return fail(h, DNATOK_ERR_STATE, "a stream is open on this handle");
    if (!id_offsets_d || offsets_capacity < 1 || !ids_out_d)
        return fail(h, DNATOK_ERR_ARG, "ids_out and id_offsets are required");
    if (((uintptr_t)id_offsets_d & 7u) || ((uintptr_t)ids_out_d & 3u))
        return fail(h, DNATOK_ERR_ARG, "misaligned output arrays");
    if (before && (before->nb < 0 || before->d < 0 || before->t < 0 || before->h < 0 ||
                   before->line_state > HS_SQ))
        return fail(h, DNATOK_ERR_ARG, "malformed part state");
    if (ids_capacity < n + 1) return fail(h, DNATOK_ERR_CAPACITY, "ids_out needs n + 1 entries");
    dnatok_status st = part_scratch(h);
    if (st != DNATOK_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int mode = (h->mode == DNATOK_CHAR) ? MODE_CHAR : MODE_KMER;
    const int k = (mode == MODE_CHAR) ? 1 : h->k;
    const int eb = last ? 1 : 0;
    if (before && before->nb == 0 && n == 0 && !eb) {  // an empty part changes nothing
        *after = *before;
        return DNATOK_OK;
    }
    Carry c;
    if (!before || before->nb > 0) {
        // the real encode of a part: from the stream start, or from the
        // state of everything before it
        if (before) {
            const Carry cb = to_carry(*before);
            cudaError_t e = cudaMemcpyAsync(part_carry(h), &cb, sizeof(Carry), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemcpyAsync(part state)");
        }
        st = part_run(h, mode, k, bytes_d, n, before != nullptr, before ? before->d : 0,
                      before ? before->nb : 0, eb, ids_out_d, ids_capacity, id_offsets_d,
                      offsets_capacity, &c, s);
        if (st != DNATOK_OK) return st;
        *after = from_carry(c);
        return DNATOK_OK;
    }
    // The part's own state (before: no boundary seen, only the line state).
    // The look-back's inclusive prefixes leave out the symbols before the
    // first boundary (a prefix from the stream start always has one), so the
    // part is encoded after a boundary set at its start: the state then
    // reads nb + 1 boundaries, t, codes, and ceil(h / k) + d ids.  h itself
    // is the offset of the first real record in a run with k = 1.
    Carry fake = to_carry(*before);
    fake.a = agg_identity();
    fake.a.nb = 1;
    cudaError_t e = cudaMemcpyAsync(part_carry(h), &fake, sizeof(Carry), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemcpyAsync(part state)");
    st = part_run(h, mode, k, bytes_d, n, true, 0, 1, eb, ids_out_d, ids_capacity, id_offsets_d,
                  offsets_capacity, &c, s);
    if (st != DNATOK_OK) return st;
    long long h_sym = 0;
    if (c.a.nb > 1) {
        if (k > 1) {  // the symbol counts: the same kernel with 1-mers
            Carry c1;
            e = cudaMemcpyAsync(part_carry(h), &fake, sizeof(Carry), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemcpyAsync(part state)");
            st = part_run(h, MODE_KMER, 1, bytes_d, n, true, 0, 1, eb, ids_out_d, ids_capacity,
                          id_offsets_d, offsets_capacity, &c1, s);
            if (st != DNATOK_OK) return st;
        }
        e = cudaMemcpy(&h_sym, id_offsets_d, sizeof(long long), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemcpy(first record offset)");
    }
    dnatok_part_state out;
    out.line_state = c.hstate;
    out.pad = 0;
    out.codes = c.a.codes;
    if (c.a.nb > 1) {
        out.nb = c.a.nb - 1;
        out.h = h_sym;
        out.d = c.a.d - (h_sym + k - 1) / k;
        out.t = c.a.t;
    } else {  // no boundary in the part: every symbol is before the first
        out.nb = 0;
        out.h = c.a.t;
        out.d = 0;
        out.t = 0;
    }
    *after = out;
    return DNATOK_OK;
}

dnatok_status dnatok_part_combine(int32_t k, const dnatok_part_state *a,
                                  const dnatok_part_state *b, dnatok_part_state *out) {
    if (k < 1 || k > DNATOK_MAX_K || !a || !b || !out) return DNATOK_ERR_ARG;
    const Carry ca = to_carry(*a), cb = to_carry(*b);
    Carry r;
    r.a = host_combine(ca.a, cb.a, k);
    r.hstate = cb.hstate;
    r.pad = 0;
    *out = from_carry(r);
    return DNATOK_OK;
}

}  // extern "C"
