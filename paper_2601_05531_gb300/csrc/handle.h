// handle.h -- the tokenizer handle behind the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

struct StreamState;  // host-streamed pipeline (stream.cu)
struct BpeState;     // BPE tables and workspace (bpe.cu)
struct OvlState;     // overlapping k-mer workspace (ovl.cu)
struct FastaState;   // compacted FASTA workspace (fasta.cu)

struct dnatok_handle {
    int mode = 0;
    int k = 1;
    int fmt = 0;
    int device = 0;
    int sm_count = 0;

    int32_t lut_host[256];
    int *d_lut = nullptr;  // CHAR table on the device

    // look-back workspace (grows on demand)
    dnatok::TileDesc *d_desc = nullptr;
    long long desc_cap = 0;
    int *d_tile_rec = nullptr;
    long long rec_cap = 0;
    unsigned long long *d_counter = nullptr;
    int *d_status = nullptr;
    unsigned *d_gate = nullptr;  // direct path -> general path switch (an epoch)
    unsigned epoch = 0;

    long long spin_limit = dnatok::kSpinLimit;  // polls of a look-back wait (dnatok_set_wait_limit)
    long long skip_chunk = -1;                  // next launch only (dnatok_inject_lookback_stall)

    dnatok::LaunchShape shape{16384, 256, 4, 8};
    dnatok::DirectShape dshape{2, 4, 0};  // direct k-mer kernel (dnatok_set_direct_launch)
    unsigned direct_epoch = 0;  // the epoch of the last encode that tried the direct path, or 0
    // dnatok_set_kernel_timing: events around the direct k-mer kernel
    cudaEvent_t ktime[2] = {nullptr, nullptr};
    bool ktime_on = false;
    bool ktime_valid = false;  // the events hold the last such launch
    bool direct = true;  // try the direct path on RAW input (dnatok_set_direct)  // tile, threads, CTAs per SM, tiles per chunk

    // device staging of dnatok_encode_host
    uint8_t *d_stage_bytes = nullptr;
    long long stage_bytes_cap = 0;
    long long *d_stage_offs = nullptr;
    long long stage_offs_cap = 0;
    long long *d_stage_out_offs = nullptr;
    long long stage_out_offs_cap = 0;
    long long *d_stage_totals = nullptr;

    StreamState *stream = nullptr;
    void *d_part = nullptr;  // parts of a split stream: carries, newline scan, map, totals (part.cu)
    BpeState *bpe = nullptr;
    OvlState *ovl = nullptr;
    FastaState *fasta = nullptr;

    // table-driven k-mers: kmer_lut (5^k ids) on the device, the single-symbol ids
    int32_t *d_klut = nullptr;
    uint16_t *d_klut16 = nullptr;  // the same as u16 (0xFFFF = none) when k <= 6 and ids < 0xFFFF
    bool kent16 = false;           // k <= 6, every kmer_lut id below 0x8000 (2-byte window entries)
    std::vector<int32_t> klut_host;
    int32_t base_ids[5] = {0, 1, 2, 3, 4};
    std::vector<int32_t> merges_host;  // BPE table, kept for the decode table

    // decode: reverse lookup table (text of id v = text[off[v] .. off[v+1])),
    // built at the first dnatok_decode; dec_v < 0 until then
    int32_t *d_dec_off = nullptr;
    uint8_t *d_dec_text = nullptr;
    long long dec_v = -1;
    int dec_max_len = 0;
    // per-tile sums of the decode passes
    long long *d_dsum = nullptr;
    long long *d_dinv = nullptr;
    long long dsum_cap = 0;

    std::string last_error;
};

namespace dnatok {

// Set the handle's (or the thread's) last error text and return `st`.
dnatok_status fail(dnatok_handle *h, dnatok_status st, const std::string &msg);
dnatok_status fail_cuda(dnatok_handle *h, cudaError_t e, const char *what);

// Grow the look-back workspace for n_bytes of input with n_bnd boundaries in
// the list (RAW); allocates (synchronously) only when it must grow.
dnatok_status ensure_workspace(dnatok_handle *h, long long n_bytes, long long n_bnd,
                               const LaunchShape &sh, cudaStream_t s);

// Next launch epoch (descriptors are reset when the 18-bit descriptor epoch
// wraps, the gate when the 32-bit epoch does).
dnatok_status next_epoch(dnatok_handle *h, cudaStream_t s, unsigned *epoch);

long long tiles_for(long long n_bytes, int head_pad, int tile);

// Launch the tile kernel over one chunk (the CHAR / KMER / SYM core).
dnatok_status run_tile_encode(dnatok_handle *h, int mode, int k, int bsrc, const uint8_t *bytes,
                              long long n_bytes, const long long *seq_offsets, long long n_bnd,
                              void *out, long long out_cap, long long *offsets_out,
                              long long offsets_cap, long long *totals_out, const Carry *carry_in,
                              Carry *carry_out, int start_boundary, int end_boundary,
                              cudaStream_t s, unsigned gate_epoch = 0);

// Direct path for RAW input without separators (direct.cu)
bool direct_eligible(int mode, long long n_seq, const int32_t *lut_host);
cudaError_t launch_direct(int mode, const uint8_t *bytes, long long n, const long long *so,
                          long long n_seq, void *out, long long *offsets_out,
                          long long *totals_out, unsigned *gate, unsigned epoch, int k,
                          const int *lut, int sm_count, const DirectShape &shape,
                          cudaStream_t s, const long long *dyn = nullptr,
                          long long out_cap = 0x7fffffffffffffffll,
                          cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
// The direct plan alone for table-driven k-mers: window offsets ceil(L / k)
// into wpre (n_seq + 1), and for every tile of 2^tile_shift windows the
// record of its first window (tile_cap entries at most).  Malformed offsets
// raise the gate instead.
cudaError_t launch_window_plan(const long long *so, long long n_seq, long long n, int k,
                               long long *wpre, long long *tile_rec, long long tile_cap,
                               int tile_shift, unsigned *gate, unsigned epoch, cudaStream_t s);

// Table-driven k-mers straight from RAW bytes without separators
// (ktab_direct.cu): the window plan, count, scan and expand; the count
// raises the gate (epoch) when the input holds a byte below 0x21.
// ktab_direct_tiles(n) entries for tile_rec and tsum;
// ktab_direct_entries(n, n_seq, k) window entries of 2 bytes (kent16) or 4.
long long ktab_direct_tiles(long long n_bytes);
long long ktab_direct_entries(long long n_bytes, long long n_seq, int k);
cudaError_t ktab_direct_setup(dnatok_handle *h);
cudaError_t ktab_direct_launch(dnatok_handle *h, const uint8_t *bytes, long long n,
                               const long long *so, long long n_seq, long long *wpre,
                               long long *tile_rec, long long *tsum, void *went, int32_t *out,
                               long long ids_cap, long long *id_offsets, long long *totals,
                               unsigned epoch, cudaStream_t s);

void fasta_destroy(dnatok_handle *h);
dnatok_status fasta_reserve(dnatok_handle *h, long long n_bytes, long long offsets_cap,
                            cudaStream_t s);
bool fasta_direct_eligible(const dnatok_handle *h, int mode, int k, const uint8_t *bytes,
                           long long n);
dnatok_status fasta_direct(dnatok_handle *h, const uint8_t *bytes, long long n, void *out,
                           long long out_cap, long long *offsets_out, long long offsets_cap,
                           long long *totals_out, const Carry *carry_in, Carry *carry_out,
                           int start_boundary, int end_boundary, unsigned epoch, int k,
                           cudaStream_t s);

// BPE path (bpe.cu)
dnatok_status bpe_create(dnatok_handle *h, const int32_t *merges, int32_t n_merges);
void bpe_destroy(dnatok_handle *h);
dnatok_status bpe_reserve(dnatok_handle *h, long long max_bytes);
dnatok_status bpe_set_launch(dnatok_handle *h, int seg_symbols, int halo);
dnatok_status bpe_get_launch(const dnatok_handle *h, int *seg_symbols, int *halo);
// {symbols, segments, segments that went through the exact repair} of the
// last encode (synchronizes the stream)
dnatok_status bpe_stats(dnatok_handle *h, long long *out, cudaStream_t s);
dnatok_status bpe_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                         const int64_t *seq_offsets_d, int64_t n_seq, int32_t *ids_out_d,
                         int64_t ids_capacity, int64_t *id_offsets_d, int64_t offsets_capacity,
                         int64_t *totals_d, cudaStream_t s);

// overlapping and table-driven k-mers on the symbol pass (ovl.cu)
void ovl_destroy(dnatok_handle *h);
dnatok_status ovl_reserve(dnatok_handle *h, long long max_bytes, long long max_offsets,
                          cudaStream_t s);
dnatok_status ovl_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                         const int64_t *seq_offsets_d, int64_t n_seq, int32_t *ids_out_d,
                         int64_t ids_capacity, int64_t *id_offsets_d, int64_t offsets_capacity,
                         int64_t *totals_d, cudaStream_t s);
dnatok_status ktab_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                          const int64_t *seq_offsets_d, int64_t n_seq, int32_t *ids_out_d,
                          int64_t ids_capacity, int64_t *id_offsets_d, int64_t offsets_capacity,
                          int64_t *totals_d, cudaStream_t s);

// Exclusive scan of per-tile sums in place, one block of kTileScanThreads
// (ovl.cu).  n_items items in tiles of items_per_tile; keys (n_rec + 1
// non-decreasing item offsets of the records) give the records with no item
// left (keys[r] >= n_items), whose rec_out entries get the total.
// totals_out (NULL or 2): {total, sum of tinv (NULL: n_rec)}.  n_rec comes
// from n_rec_dev when not NULL; n_items from n_items_dev when not NULL, else
// n_items_host when >= 0, else keys[n_rec].  Does nothing once the device
// status word holds an error.  With gate not NULL it runs only when the gate
// is raised (*gate == gate_epoch) if run_if_raised, only when it is not
// otherwise: behind a direct path it is the general path's scan, which runs
// only when the direct path declined; inside a direct path it is that
// path's own scan, which must not read what a declined plan left unwritten.
__global__ void tile_scan_kernel(long long *tsum, const long long *tinv, const long long *keys,
                                 const long long *n_rec_dev, long long n_rec_host,
                                 const long long *n_items_dev, long long n_items_host,
                                 int items_per_tile, long long *rec_out, long long *totals_out,
                                 const int *status, const unsigned *gate, unsigned gate_epoch,
                                 bool run_if_raised);
constexpr int kTileScanThreads = 1024;

// decode tables (decode.cu)
void dec_destroy(dnatok_handle *h);

// host-streamed pipeline (stream.cu)
void stream_destroy(dnatok_handle *h);

// parts of a split stream (part.cu)
void part_destroy(dnatok_handle *h);

}  // namespace dnatok
