// common.cuh -- device-side building blocks shared by the library's kernels:
// inline-PTX wrappers (TMA bulk copy, mbarrier, acquire/release), the scan
// element of the decoupled look-back, and bounded waits.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dnatok {

// ---------------------------------------------------------------- constants

enum : int { MODE_CHAR = 0, MODE_KMER = 1, MODE_BPE = 2, MODE_SYM = 3 };
enum : int { FMT_RAW = 0, FMT_FASTA = 1 };

// Device status word values (written by kernels, read by the host).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD_OFFSETS = 2, DEV_CAPACITY = 3 };

// Byte class bits of the 256-entry class table.
//   bits 0-1  base code (A0 C1 G2 T3)    bit 2  N-class
//   bit 3     separator (\n \r space \t) bit 4  '\n'    bit 5  '>'
enum : uint8_t { CB_N = 4, CB_SEP = 8, CB_NL = 16, CB_GT = 32 };

// Look-back descriptor flags.
enum : unsigned { LB_EMPTY = 0, LB_AGG = 1, LB_INCL = 2 };

// FASTA line states.
enum : unsigned { HS_LS = 0, HS_HD = 1, HS_SQ = 2 };

// A bounded spin: about this many polls (each followed by a short sleep)
// before a wait gives up, records DEV_TIMEOUT and returns.
constexpr int kSpinLimit = 1 << 22;

// ------------------------------------------------------------ scan element
//
// Scan element over a span of the byte stream (the monoid of the single-pass
// look-back).  Boundaries are record starts (and the end of the stream).
//   nb    boundaries inside the span
//   h     kept symbols before the first boundary (all kept symbols if nb == 0)
//   d     tokens completed after the first boundary: ceil(L/k) for every
//         record closed inside the span, floor(t/k) for the record still open
//   t     kept symbols after the last boundary (0 if nb == 0)
//   codes the last min(open, k-1) kept symbols of the open record, 3 bits each
//         (base code in bits 0-1, N flag in bit 2), newest in the low bits;
//         symbol count in bits 58..61.
// An exclusive prefix from the stream start always has nb >= 1 (position 0
// is a boundary), so it reads: records seen = nb, tokens completed = d,
// kept symbols of the open record = t.
struct Agg {
    long long nb, h, d, t;
    unsigned long long codes;
};

__host__ __device__ __forceinline__ Agg agg_identity() { return Agg{0, 0, 0, 0, 0ull}; }

__host__ __device__ __forceinline__ int codes_count(unsigned long long c) { return (int)(c >> 58); }

__host__ __device__ __forceinline__ unsigned long long codes_concat(unsigned long long a,
                                                                   unsigned long long b, int k) {
    if (k <= 1) return 0ull;
    int na = codes_count(a), nb = codes_count(b);
    int n = na + nb;
    if (n > k - 1) n = k - 1;
    const unsigned long long m58 = (1ull << 58) - 1;
    unsigned long long bits = ((a & m58) << (3 * nb)) | (b & m58);
    bits &= (n == 0) ? 0ull : ((1ull << (3 * n)) - 1);
    return ((unsigned long long)n << 58) | bits;
}

// Division by the k-mer length without a division instruction sequence:
// floor(x / k) = high 64 bits of x * ceil(2^64 / k), exact for x < 2^44
// (the error term x / 2^64 stays below the gap 1/k between fractions).
struct KDiv {
    int k;
    unsigned long long m64;  // ceil(2^64 / k), k >= 2
    unsigned m32;            // ceil(2^32 / k), k >= 2: exact for x < 2^17
    __device__ __forceinline__ long long div(long long x) const {
        return k == 1 ? x : (long long)__umul64hi((unsigned long long)x, m64);
    }
    __device__ __forceinline__ unsigned div32(unsigned x) const {
        return k == 1 ? x : __umulhi(x, m32);
    }
};

__device__ __forceinline__ KDiv make_kdiv(int k) {
    KDiv d;
    d.k = k;
    d.m64 = k > 1 ? ~0ull / (unsigned long long)k + 1ull : 0ull;
    d.m32 = k > 1 ? (unsigned)((0x100000000ull + (unsigned long long)k - 1) / (unsigned long long)k) : 0u;
    return d;
}

__device__ __forceinline__ Agg agg_combine(const Agg &A, const Agg &B, const KDiv &kd) {
    const int k = kd.k;
    Agg r;
    r.nb = A.nb + B.nb;
    if (A.nb == 0) {
        r.h = A.h + B.h;
        r.d = B.d;
        r.t = B.t;
    } else if (B.nb == 0) {
        r.h = A.h;
        r.d = A.d - kd.div(A.t) + kd.div(A.t + B.h);
        r.t = A.t + B.h;
    } else {
        r.h = A.h;
        r.d = A.d - kd.div(A.t) + kd.div(A.t + B.h + k - 1) + B.d;
        r.t = B.t;
    }
    r.codes = (B.nb > 0) ? B.codes : codes_concat(A.codes, B.codes, k);
    return r;
}

// Carry between consecutive chunks of one stream: the inclusive prefix at the
// chunk end plus the FASTA line state there.
struct Carry {
    Agg a;
    unsigned hstate;
    unsigned pad;
};

// One look-back descriptor per tile: four 64-bit words that first hold the
// tile's own scan element (flag LB_AGG) and are then overwritten by the
// inclusive prefix through the tile (flag LB_INCL).  Every word carries a tag
// (18-bit launch epoch, 2-bit flag) in its top 20 bits and a 44-bit value
// below, so status and payload arrive in one round trip and a reader that
// catches the overwrite half done sees mixed tags and simply polls again.
//   aggregate: nb | (h << 22 | d) | t | codes   (h, d < 2^22: tile-local)
//   inclusive: nb | d | t | codes               (h = 0: a prefix from the
//                                                stream start opens at a
//                                                boundary)
// The k-mer symbol count of `codes` is not stored: it equals
// min(open symbols, k - 1), open = (nb > 0 ? t : h).
struct __align__(64) TileDesc {
    unsigned long long w[4];
    unsigned hstatus;  // FASTA line-state map: epoch << 8 | flag << 6 | map
    unsigned pad[7];
};

constexpr unsigned long long kValMask = (1ull << 44) - 1;
constexpr unsigned kEpochBits = 18;

__host__ __device__ __forceinline__ unsigned desc_tag(unsigned epoch, unsigned flag) {
    return ((epoch & ((1u << kEpochBits) - 1)) << 2) | flag;
}

__host__ __device__ __forceinline__ int codes_open_count(const Agg &a, int k) {
    const long long open = a.nb > 0 ? a.t : a.h;
    return (int)(open < k - 1 ? open : (k - 1 > 0 ? k - 1 : 0));
}

// ---------------------------------------------------------------- PTX

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_try_wait, but the thread may be suspended (issuing nothing) for up
// to hint_ns nanoseconds while the phase is incomplete.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, unsigned parity, unsigned hint_ns) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// 1-D TMA bulk copy global -> shared, completion counted on an mbarrier.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *smem_dst, const void *gsrc, unsigned bytes,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 1-D TMA bulk copy shared -> global (bulk-group completion).  Both
// addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_store_1d(void *gdst, const void *ssrc, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_addr(ssrc)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until this thread's bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Wait until this thread's bulk stores are complete.
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long ld_relaxed_s64(const long long *p) {
    long long v;
    asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_s64(long long *p, long long v) {
    asm volatile("st.relaxed.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_v2u64(unsigned long long *p, unsigned long long a,
                                                 unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b)
                 : "memory");
}
__device__ __forceinline__ void ld_relaxed_v2u64(const unsigned long long *p,
                                                 unsigned long long &a, unsigned long long &b) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p)
                 : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Publish a tile's scan element (LB_AGG) or inclusive prefix (LB_INCL).
__device__ __forceinline__ void publish_desc(TileDesc *d, const Agg &a, unsigned epoch,
                                             unsigned flag) {
    const unsigned long long tg = (unsigned long long)desc_tag(epoch, flag) << 44;
    const unsigned long long w1 = (flag == LB_AGG)
                                      ? (((unsigned long long)a.h << 22) | (unsigned long long)a.d)
                                      : (unsigned long long)a.d;
    st_relaxed_v2u64(d->w, tg | ((unsigned long long)a.nb & kValMask), tg | (w1 & kValMask));
    st_relaxed_v2u64(d->w + 2, tg | ((unsigned long long)a.t & kValMask),
                     tg | (a.codes & kValMask));
}
// Decode four words read from a descriptor: LB_AGG / LB_INCL, or LB_EMPTY
// when they are stale (another epoch) or torn (mixed tags).
__device__ __forceinline__ unsigned decode_desc(unsigned long long w0, unsigned long long w1,
                                                unsigned long long w2, unsigned long long w3,
                                                unsigned epoch, int k, Agg &a) {
    const unsigned tg = (unsigned)(w0 >> 44);
    if ((unsigned)(w1 >> 44) != tg || (unsigned)(w2 >> 44) != tg || (unsigned)(w3 >> 44) != tg)
        return LB_EMPTY;
    if ((tg >> 2) != (epoch & ((1u << kEpochBits) - 1))) return LB_EMPTY;
    const unsigned flag = tg & 3u;
    if (flag != LB_AGG && flag != LB_INCL) return LB_EMPTY;
    a.nb = (long long)(w0 & kValMask);
    if (flag == LB_AGG) {
        a.h = (long long)((w1 & kValMask) >> 22);
        a.d = (long long)(w1 & ((1ull << 22) - 1));
    } else {
        a.h = 0;
        a.d = (long long)(w1 & kValMask);
    }
    a.t = (long long)(w2 & kValMask);
    a.codes = ((unsigned long long)codes_open_count(a, k) << 58) | (w3 & kValMask);
    return flag;
}

__device__ __forceinline__ Agg load_agg(const Agg *p) {
    const long long *q = reinterpret_cast<const long long *>(p);
    Agg a;
    a.nb = ld_relaxed_s64(q + 0);
    a.h = ld_relaxed_s64(q + 1);
    a.d = ld_relaxed_s64(q + 2);
    a.t = ld_relaxed_s64(q + 3);
    a.codes = (unsigned long long)ld_relaxed_s64(q + 4);
    return a;
}

__device__ __forceinline__ void store_agg(Agg *p, const Agg &a) {
    long long *q = reinterpret_cast<long long *>(p);
    st_relaxed_s64(q + 0, a.nb);
    st_relaxed_s64(q + 1, a.h);
    st_relaxed_s64(q + 2, a.d);
    st_relaxed_s64(q + 3, a.t);
    st_relaxed_s64(q + 4, (long long)a.codes);
}

__device__ __forceinline__ Agg shfl_up_agg(const Agg &a, int o) {
    Agg r;
    r.nb = __shfl_up_sync(0xffffffffu, a.nb, o);
    r.h = __shfl_up_sync(0xffffffffu, a.h, o);
    r.d = __shfl_up_sync(0xffffffffu, a.d, o);
    r.t = __shfl_up_sync(0xffffffffu, a.t, o);
    r.codes = __shfl_up_sync(0xffffffffu, a.codes, o);
    return r;
}

__device__ __forceinline__ Agg shfl_agg(const Agg &a, int src) {
    Agg r;
    r.nb = __shfl_sync(0xffffffffu, a.nb, src);
    r.h = __shfl_sync(0xffffffffu, a.h, src);
    r.d = __shfl_sync(0xffffffffu, a.d, src);
    r.t = __shfl_sync(0xffffffffu, a.t, src);
    r.codes = __shfl_sync(0xffffffffu, a.codes, src);
    return r;
}

// Record an error in the device status word (first error wins).
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while the previous kernel on its
// stream is still running; pdl_wait() blocks until that kernel has finished
// and its memory is visible (a no-op otherwise); pdl_launch_dependents() lets
// the next such kernel start early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void set_dev_status(int *status, int code) {
    if (status) atomicCAS(status, DEV_OK, code);
}

__device__ __forceinline__ bool dev_failed(const int *status) {
    return status && *((volatile const int *)status) != DEV_OK;
}

// FASTA line-state maps: a map sends each of the three states (LS, HD, SQ) to
// a state, 2 bits per entry.  compose(f, g) applies f first, then g.
__host__ __device__ __forceinline__ unsigned hmap_apply(unsigned m, unsigned s) {
    return (m >> (2 * s)) & 3u;
}
__host__ __device__ __forceinline__ unsigned hmap_compose(unsigned f, unsigned g) {
    return hmap_apply(g, hmap_apply(f, 0)) | (hmap_apply(g, hmap_apply(f, 1)) << 2) |
           (hmap_apply(g, hmap_apply(f, 2)) << 4);
}
constexpr unsigned kHmapIdentity = 0u | (1u << 2) | (2u << 4);
__host__ __device__ __forceinline__ unsigned hmap_const(unsigned s) {
    return s | (s << 2) | (s << 4);
}
// One byte of the FASTA line-state machine.
__host__ __device__ __forceinline__ unsigned hstep(unsigned s, uint8_t b) {
    if (b == '\n') return HS_LS;
    if (s == HS_LS) return b == '>' ? HS_HD : HS_SQ;
    return s;
}

}  // namespace dnatok
