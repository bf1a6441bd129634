/*
 * dnatok.h -- C ABI of the GB300 DNA byte -> token-ID library (libdnatok.so).
 *
 * The library turns raw DNA bytes into token-ID streams on one GPU, following
 * the problem statement of Niktab & Patel, "DNATokenizer: A GPU-First
 * Byte-to-Identifier Tokenizer" (arXiv 2601.05531): bytes go to the device
 * and a device-resident byte -> identifier table is applied there (Sec. 2.2,
 * "Bytes path"; Algorithm 2), producing the integer identifiers that an
 * embed_tokens : Z^{B x T} -> R^{B x T x D} consumes (Sec. 2).  Sequences
 * here are ragged (one flat byte array plus offsets) instead of the paper's
 * equal-length B x T matrix, and FASTA text is accepted directly.
 *
 * Tokenization modes (Sec. 1.1, Table 1; Sec. 1.3 lists all three):
 *   DNATOK_CHAR  single-nucleotide: id = lut[byte] (Algorithm 1's ascii_lut);
 *   DNATOK_KMER  non-overlapping k-mers, id = sum_i 4^(k-1-i) * code(b_i),
 *                A0 C1 G2 T3, UNK = 4^k (MapKmer, Algorithm 2);
 *   DNATOK_BPE   greedy rank-ordered BPE merges of a fixed table
 *                (segmentation identical to the table's tokenizer, Sec. 4.3);
 *   DNATOK_KMER_OVERLAP  overlapping k-mers (window step 1): a token at every
 *                kept base j with j + k <= L of a record of L kept bases
 *                (L - k + 1 tokens, none when L < k; Sec. 1.1, Table 1), same
 *                ids and UNK as DNATOK_KMER.  One-shot encodes only (no
 *                host streams, no serving loop).
 *   DNATOK_KMER_TABLE  table-driven non-overlapping k-mers (Algorithm 1
 *                builds kmer_lut[0..5^k-1] over base-5 digits A0 C1 G2 T3
 *                N4 and Algorithm 2 applies it as MapKmer): each whole window
 *                of k kept symbols emits kmer_lut[sum_i 5^(k-1-i) d_i] when
 *                that entry is >= 0, otherwise its k symbols one by one as
 *                base_ids[d]; a tail of L mod k symbols emits base_ids[d]
 *                for each.  1 <= k <= 10.  One-shot encodes only.
 *
 * Conventions for what the paper leaves open (identical in the CPU oracle):
 *   - case-insensitive; '\n' '\r' ' ' '\t' are dropped (they emit nothing and
 *     do not move the k-mer frame; BPE words continue across them);
 *   - every other non-ACGT byte is N-class: CHAR default id 4, k-mer UNK,
 *     BPE: ends the word and emits N_ID = 4 + n_merges;
 *   - a k-mer tail of L mod k > 0 bases emits one UNK;
 *   - CHAR default table: A0 C1 G2 T3, N-class 4, separators -1 (dropped);
 *   - BPE ids: bases 0..3, merge rank r -> 4 + r;
 *   - FASTA: a line whose first byte is '>' is a header; it is dropped with
 *     its newline and opens a record; bytes before the first header form a
 *     record only when byte 0 is not '>'.
 *
 * Output layout: ids are int32, packed record after record with no padding;
 * id_offsets (int64) has one entry per record boundary, so record r's ids are
 * ids[id_offsets[r] .. id_offsets[r+1]).
 *
 * Threading: a handle may be used by one host thread at a time, and its
 * device work must stay ordered on one CUDA stream at a time (its
 * look-back descriptors are reused by every launch).  Handles are
 * independent of each other.
 *
 * Errors: every entry point returns a dnatok_status.  Argument and table
 * errors are reported synchronously.  Launches are asynchronous; a device-side
 * error (a bounded wait that ran out, malformed device offsets) is recorded in
 * the handle and reported by dnatok_sync() or by the next call that
 * synchronizes; dnatok_last_error() gives the text of the last error.
 */
#ifndef DNATOK_H
#define DNATOK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DNATOK_API __attribute__((visibility("default")))
#else
#define DNATOK_API
#endif

typedef enum {
    DNATOK_OK = 0,
    DNATOK_PENDING = 1,           /* request not finished yet (poll again) */
    DNATOK_ERR_ARG = -1,          /* bad argument (null, negative size, k out of range ...) */
    DNATOK_ERR_TABLE = -2,        /* invalid LUT or merge table */
    DNATOK_ERR_CAPACITY = -3,     /* an output buffer is too small */
    DNATOK_ERR_CUDA = -4,         /* a CUDA runtime call failed */
    DNATOK_ERR_BUDGET = -5,       /* request larger than the device-memory budget */
    DNATOK_ERR_TIMEOUT = -6,      /* a bounded device-side wait ran out */
    DNATOK_ERR_UNKNOWN_REQ = -7,  /* no such request id */
    DNATOK_ERR_NOMEM = -8,        /* host or device allocation failed */
    DNATOK_ERR_STATE = -9,        /* call not valid in the current state */
    DNATOK_ERR_DEVICE_DATA = -10  /* device-side input (seq_offsets) malformed */
} dnatok_status;

typedef enum {
    DNATOK_CHAR = 0,
    DNATOK_KMER = 1,
    DNATOK_BPE = 2,
    DNATOK_KMER_OVERLAP = 3,
    DNATOK_KMER_TABLE = 4
} dnatok_mode;
typedef enum { DNATOK_RAW = 0, DNATOK_FASTA = 1 } dnatok_format;

/* Same type as cudaStream_t (NULL = the legacy default stream). */
typedef struct CUstream_st *dnatok_cuda_stream;

typedef struct dnatok_handle dnatok_handle;

/* Tables, copied by dnatok_create (the caller keeps ownership of its arrays).
 *   ascii_lut256: CHAR only; 256 host int32 ids, -1 = drop the byte; NULL =
 *                 default table.  Ids must be >= -1.  This is the ascii_lut of
 *                 Algorithm 1 (e.g. its fixed DNA fallback A1 C2 G3 T4 N0).
 *   merges:       BPE only; n_merges host (left, right) int32 pairs in rank
 *                 order.  Valid iff for every rank r both ids are < 4 + r and
 *                 no pair repeats.  n_merges <= DNATOK_MAX_MERGES.
 *   kmer_lut:     DNATOK_KMER_TABLE only; 5^k host int32 ids indexed by
 *                 sum_i 5^(k-1-i) d_i (digits A0 C1 G2 T3, N-class 4), each
 *                 >= -1; -1 = no entry (the window falls back to base_ids).
 *   base_ids:     DNATOK_KMER_TABLE only; 5 host int32 ids >= 0 for the
 *                 single symbols A C G T N. */
typedef struct {
    const int32_t *ascii_lut256;
    const int32_t *merges;
    int32_t n_merges;
    const int32_t *kmer_lut;
    const int32_t *base_ids;
} dnatok_tables;

#define DNATOK_MAX_K 15
#define DNATOK_MAX_K_TABLE 10
#define DNATOK_MAX_MERGES 16384

/* Create a tokenizer on the current CUDA device.  mode/k/tables as above (k
 * is ignored unless mode is DNATOK_KMER, DNATOK_KMER_OVERLAP (1 <= k <= 15)
 * or DNATOK_KMER_TABLE (1 <= k <= 10)).  fmt selects how
 * records are found by dnatok_encode and the stream API.  Tables are
 * validated and copied to device memory.  On success *out owns its device
 * tables and workspace; release it with dnatok_destroy. */
DNATOK_API dnatok_status dnatok_create(dnatok_handle **out, dnatok_mode mode, int k,
                            const dnatok_tables *tables, dnatok_format fmt);

/* Free everything the handle owns.  Waits for its outstanding device work. */
DNATOK_API void dnatok_destroy(dnatok_handle *h);

/* Upper bound on the ids produced from n_bytes of input in n_seq records
 * (RAW) -- use it to size ids_out.  FASTA: n_seq is ignored. */
DNATOK_API dnatok_status dnatok_max_tokens(const dnatok_handle *h, int64_t n_bytes, int64_t n_seq,
                                int64_t *cap);

/* Reserve device workspace for inputs up to max_bytes / max_seq so that later
 * dnatok_encode calls of that size allocate nothing (needed before stream
 * capture).  Synchronizes the device if it grows. */
DNATOK_API dnatok_status dnatok_reserve(dnatok_handle *h, int64_t max_bytes, int64_t max_seq);

/*
 * One-shot encode, asynchronous on `stream` (every pointer is DEVICE memory
 * owned by the caller and must stay valid until the stream reaches this work).
 *   bytes_d        n_bytes input bytes (any alignment).
 *   seq_offsets_d  RAW: n_seq + 1 non-decreasing int64 with [0] = 0 and
 *                  [n_seq] = n_bytes; record r = bytes[off[r] .. off[r+1]).
 *                  Checked on the device (DNATOK_ERR_DEVICE_DATA via
 *                  dnatok_sync).  FASTA: ignored (pass NULL, 0).
 *   ids_out_d      capacity ids_capacity >= dnatok_max_tokens(n_bytes, n_seq),
 *                  checked here (DNATOK_ERR_CAPACITY).  Entries after the ids
 *                  produced, up to the capacity, are scratch: a direct path
 *                  that finds its premise broken may leave ids there before
 *                  the general path rewrites the result.
 *   id_offsets_d   RAW: n_seq + 1 entries.  FASTA: offsets_capacity entries;
 *                  the records found may exceed it: entries past the capacity
 *                  are not written and totals tells how many there were.
 *   totals_d       NULL or 2 int64: {number of ids, number of records}.
 * Workspace (look-back descriptors) is owned by the handle; it grows with a
 * synchronizing allocation when n_bytes exceeds what was reserved.
 */
DNATOK_API dnatok_status dnatok_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                            const int64_t *seq_offsets_d, int64_t n_seq, int32_t *ids_out_d,
                            int64_t ids_capacity, int64_t *id_offsets_d,
                            int64_t offsets_capacity, int64_t *totals_d,
                            dnatok_cuda_stream stream);

/*
 * Encode from HOST buffers (the end-to-end form): copies host_bytes and
 * host_seq_offsets (RAW) into device staging owned by the handle, runs the
 * same kernels as dnatok_encode, and copies the record offsets and totals
 * back to the HOST arrays id_offsets_host / totals_host (2 int64, may be
 * NULL).  The ids stay on the device in ids_out_d (the input of an embedding
 * lookup).  Page-locked (pinned) host buffers give full link bandwidth.
 * Returns when the results are on the host (it synchronizes `stream`).
 */
DNATOK_API dnatok_status dnatok_encode_host(dnatok_handle *h, const uint8_t *host_bytes,
                                            int64_t n_bytes, const int64_t *host_seq_offsets,
                                            int64_t n_seq, int32_t *ids_out_d,
                                            int64_t ids_capacity, int64_t *id_offsets_host,
                                            int64_t offsets_capacity, int64_t *totals_host,
                                            dnatok_cuda_stream stream);

/* Wait for `stream`, then report any device-side error recorded by this
 * handle's kernels (clearing it). */
DNATOK_API dnatok_status dnatok_sync(dnatok_handle *h, dnatok_cuda_stream stream);

/* Copy the text of the handle's last error into buf (always NUL-terminated).
 * h may be NULL for errors of dnatok_create. */
DNATOK_API dnatok_status dnatok_last_error(const dnatok_handle *h, char *buf, size_t len);

/* ------------------------------------------------------- host-streamed */

/*
 * Host-streamed encode: the bytes path's pinned staging with the pipelined
 * path's two streams, so that the copy of one chunk overlaps the
 * tokenization of the previous one (Sec. 2.2 "Encoding paths"; the overlap
 * on/off ablation of Sec. 3.5 and the crossover of Sec. 4.2).  The caller feeds one logical byte stream in pieces of
 * any size; the handle cuts them into chunks, copies each chunk into a ring
 * of device slots on a copy stream and tokenizes it on a compute stream,
 * carrying the scan state (open record, partial k-mer, FASTA line state)
 * from chunk to chunk, so that the result equals dnatok_encode of the whole
 * stream.  Ids and record offsets are written at their global positions in
 * the caller's DEVICE arrays given to dnatok_stream_open.
 *
 * Records: FASTA handles find them as dnatok_encode does.  RAW handles: the
 * first piece opens record 0, a piece flagged DNATOK_NEW_RECORD opens the
 * next record, DNATOK_END_OF_STREAM closes the last one; no more pieces may
 * follow it.  Not available for DNATOK_BPE handles (DNATOK_ERR_STATE).
 * While a stream is open the handle runs nothing else.
 */
#define DNATOK_END_OF_STREAM 1 /* this piece ends the stream */
#define DNATOK_NEW_RECORD 2    /* RAW: a record starts at this piece's first byte */
#define DNATOK_HOST_PINNED 4   /* host_bytes is page-locked and stays valid until the
                                  request completes: copied by DMA straight from it */

typedef struct {
    int64_t chunk_bytes; /* bytes per chunk (0 = 64 MiB) */
    int32_t n_slots;     /* device slots in the ring, 2..8 (0 = 3) */
    int32_t overlap;     /* 1 = copies on their own stream (default); 0 = copy and
                            compute serialized on one stream (the ablation) */
} dnatok_stream_cfg;

typedef struct {
    int64_t n_ids;     /* ids written so far (whole stream through this request) */
    int64_t n_records; /* records closed so far */
    int64_t bytes_in;  /* input bytes submitted through this request */
} dnatok_stream_result;

/* Open a stream on h.  ids_out_d / id_offsets_d: caller-owned DEVICE arrays
 * that receive the whole stream's ids and record offsets; they must stay
 * valid until dnatok_stream_close.  Ids past ids_capacity are not written
 * (the poll then reports DNATOK_ERR_CAPACITY); offsets past
 * offsets_capacity are not written either (n_records still counts them).
 * Allocates the device ring (and, on first need, a page-locked host ring). */
DNATOK_API dnatok_status dnatok_stream_open(dnatok_handle *h, const dnatok_stream_cfg *cfg,
                                            int32_t *ids_out_d, int64_t ids_capacity,
                                            int64_t *id_offsets_d, int64_t offsets_capacity);

/* Queue n bytes of the stream.  Without DNATOK_HOST_PINNED the bytes are
 * copied into the page-locked ring before this returns (the caller may reuse
 * its buffer at once); with it, they are copied by DMA from host_bytes, which
 * must stay valid until the request completes.  *req_id identifies the
 * request for poll / wait. */
DNATOK_API dnatok_status dnatok_stream_submit(dnatok_handle *h, const uint8_t *host_bytes,
                                              int64_t n, int flags, uint64_t *req_id);

/* DNATOK_PENDING while the request's chunks are still in flight; DNATOK_OK
 * once its ids and offsets are on the device (out filled in);
 * DNATOK_ERR_UNKNOWN_REQ for an id never issued or more than 1024 requests
 * old; a device-side error of any chunk so far is returned here. */
DNATOK_API dnatok_status dnatok_stream_poll(dnatok_handle *h, uint64_t req_id,
                                            dnatok_stream_result *out);

/* Block until the request completes, then as dnatok_stream_poll. */
DNATOK_API dnatok_status dnatok_stream_wait(dnatok_handle *h, uint64_t req_id,
                                            dnatok_stream_result *out);

/* Wait for every request, release the ring.  The handle can open another
 * stream afterwards. */
DNATOK_API dnatok_status dnatok_stream_close(dnatok_handle *h);

/* -------------------------------------------------------------- serving */

/*
 * Serving loop: requests of mixed modes and sizes are submitted at any time
 * (host bytes, one request = one record); a worker thread admits them under a
 * device-memory budget, packs the queued requests of one mode into a batch
 * and launches it on one of n_slots streams while earlier batches still run
 * (continuous batching).  Every slot holds its own handle per mode, so the
 * tables stay resident; inputs and outputs live in one device arena of
 * budget_bytes (a request's ids stay there until it is released).  The paper
 * names serving as a target use (Sec. 4.4) without a design.
 */
typedef struct dnatok_server dnatok_server;
typedef struct {
    int64_t budget_bytes;        /* device arena: inputs + outputs of admitted requests */
    int64_t host_arena_bytes;    /* page-locked staging of submitted bytes */
    int64_t max_batch_bytes;     /* input bytes packed into one batch (also the largest request) */
    int32_t max_batch_requests;  /* requests in one batch */
    int32_t n_slots;             /* batches in flight at once (streams), 1..16 */
    int32_t kmer_k;              /* k of the DNATOK_KMER mode */
    int32_t n_merges;            /* BPE table (DNATOK_BPE mode), may be 0 */
    const int32_t *merges;
} dnatok_server_cfg;

typedef struct {
    const int32_t *ids_d;  /* device ids of the request, valid until it is released */
    int64_t n_ids;
    double latency_us;     /* submit -> completion seen by the worker */
} dnatok_server_result;

typedef struct {
    int64_t device_bytes_in_use;
    int64_t batches_launched;
    int64_t queued;
    int64_t batches_running;
} dnatok_server_counters;

/* DNATOK_ERR_ARG on a bad configuration; DNATOK_ERR_BUDGET when one request
 * of max_batch_bytes (input, worst-case ids and offsets) would not fit
 * budget_bytes on its own. */
DNATOK_API dnatok_status dnatok_server_create(const dnatok_server_cfg *cfg, dnatok_server **out);
/* Copy n host bytes into the staging arena and queue them (mode: DNATOK_CHAR
 * with the default table, DNATOK_KMER with cfg.kmer_k, DNATOK_BPE with
 * cfg.merges).  DNATOK_ERR_BUDGET if the staging arena is full (retry after
 * releasing), DNATOK_ERR_CAPACITY if n exceeds max_batch_bytes. */
DNATOK_API dnatok_status dnatok_server_submit(dnatok_server *s, int32_t mode,
                                              const uint8_t *host_bytes, int64_t n,
                                              uint64_t *req_id);
/* DNATOK_PENDING, or DNATOK_OK with the result filled in. */
DNATOK_API dnatok_status dnatok_server_poll(dnatok_server *s, uint64_t req_id,
                                            dnatok_server_result *out);
/* Copy a finished request's ids to host memory (capacity ids; *n_ids gets the
 * count; DNATOK_ERR_CAPACITY if they do not fit).  Synchronous. */
DNATOK_API dnatok_status dnatok_server_read(dnatok_server *s, uint64_t req_id, int32_t *host_ids,
                                            int64_t capacity, int64_t *n_ids);
/* Give the request's device output back to the arena. */
DNATOK_API dnatok_status dnatok_server_release(dnatok_server *s, uint64_t req_id);
DNATOK_API dnatok_status dnatok_server_stats(dnatok_server *s, dnatok_server_counters *out);
/* Failure injection, for testing how a caller handles failed requests: the
 * next `count` batches the worker launches fail -- kind 1: as if
 * dnatok_encode refused the batch on the host; kind 2: as if a kernel of the
 * batch recorded a device-side error (a bounded wait that ran out).  Every
 * request of such a batch completes with DNATOK_ERR_CUDA from poll/read;
 * the slot's handle is cleared and the batches after it run normally.
 * kind 0 cancels.  (No counterpart in the paper.) */
DNATOK_API dnatok_status dnatok_server_inject(dnatok_server *s, int32_t kind, int32_t count);
/* Stop the worker, wait for the device, free everything. */
DNATOK_API void dnatok_server_destroy(dnatok_server *s);

/* ---------------------------------------------------------------- decode */

/*
 * Token ids back to text on the device (Sec. 4, "Decode Operations", where
 * the paper leaves it as future work): a reverse lookup from each id to the
 * bases it stands for.  Per mode:
 *   DNATOK_CHAR   id v -> the first byte b with lut[b] == v in the order
 *                 "ACGTN", 'A'..'Z', 'a'..'z', then 0..255;
 *   DNATOK_KMER   id < 4^k -> its k bases (A C G T); UNK = 4^k -> one '?';
 *   DNATOK_KMER_OVERLAP  per record: the first token as DNATOK_KMER, every
 *                 later one its last base ('?' for UNK);
 *   DNATOK_BPE    the bases the merge table expands the id to; N_ID -> 'N';
 *   DNATOK_KMER_TABLE  the k digits ("ACGTN") of the smallest window index
 *                 whose kmer_lut entry is the id, else the symbol of the
 *                 smallest digit d with base_ids[d] == id.
 * An id with no inverse (out of range, PAD, a table gap) writes nothing and
 * is counted in totals_d[1].
 *   ids_d          n_ids int32 (DEVICE).
 *   id_offsets_d   n_seq + 1 non-decreasing int64 (DEVICE) with [0] = 0 and
 *                  [n_seq] = n_ids, as written by dnatok_encode; a malformed
 *                  array gives wrong record offsets but no access outside
 *                  the buffers.
 *   bytes_out_d    bytes_capacity >= dnatok_max_decoded_bytes (DEVICE;
 *                  checked here, DNATOK_ERR_CAPACITY).
 *   byte_offsets_d n_seq + 1 int64 (DEVICE): record r's text is
 *                  bytes_out[byte_offsets[r] .. byte_offsets[r+1]).
 *   totals_d       NULL or 2 int64 (DEVICE): {bytes written, ids without an
 *                  inverse}.
 * Asynchronous on `stream`.  The handle builds its inverse table at the
 * first call (synchronous upload); DNATOK_ERR_TABLE if it would exceed 2^24
 * ids or 256 MB of text.
 */
DNATOK_API dnatok_status dnatok_max_decoded_bytes(dnatok_handle *h, int64_t n_ids, int64_t n_seq,
                                                  int64_t *cap);
DNATOK_API dnatok_status dnatok_decode(dnatok_handle *h, const int32_t *ids_d, int64_t n_ids,
                                       const int64_t *id_offsets_d, int64_t n_seq,
                                       uint8_t *bytes_out_d, int64_t bytes_capacity,
                                       int64_t *byte_offsets_d, int64_t *totals_d,
                                       dnatok_cuda_stream stream);

/* ------------------------------------------------------ reverse complement */

/*
 * Reverse complement of every record (Sec. 4, "Integration with Data
 * Augmentation": the augmentation the paper leaves to future GPU work):
 * out[s + e - 1 - i] = comp(in[i]) for i in [s, e) = [seq_offsets[r],
 * seq_offsets[r+1]); comp swaps A/T, C/G, R/Y, K/M, B/V, D/H in either case
 * and keeps every other byte (S, W, N, separators, ...).  Needs no handle.
 *   bytes_d, out_d  n_bytes each (DEVICE); out must not overlap the input.
 *   seq_offsets_d   n_seq + 1 non-decreasing int64 (DEVICE), [0] = 0,
 *                   [n_seq] = n_bytes; positions a malformed array would map
 *                   outside [0, n_bytes) are left unwritten.
 * Asynchronous on `stream`; DNATOK_ERR_ARG for bad arguments.
 */
DNATOK_API dnatok_status dnatok_reverse_complement(const uint8_t *bytes_d, int64_t n_bytes,
                                                   const int64_t *seq_offsets_d, int64_t n_seq,
                                                   uint8_t *out_d, dnatok_cuda_stream stream);

/* ------------------------------------------------------- fixed-shape feed */

/*
 * Fixed-shape model feed (Algorithm 2: rows left-padded with id_pad to
 * token_len so each row's own tokens stay right-aligned; Sec. 2.2, int32
 * staging promoted on the device to the int64 an embedding call takes).
 * Row i of out (n_rows x token_len, row-major) is record row_begin + i of
 * (ids_d, id_offsets_d): a record of m <= token_len ids is written after
 * token_len - m copies of id_pad; a longer record keeps its first token_len
 * ids.  out_bytes is 4 (int32) or 8 (int64).  Needs no handle.  All
 * pointers DEVICE; asynchronous on `stream`; DNATOK_ERR_ARG for bad
 * arguments (id_pad must fit the output type).
 */
DNATOK_API dnatok_status dnatok_feed(const int32_t *ids_d, const int64_t *id_offsets_d,
                                     int64_t row_begin, int64_t n_rows, int64_t token_len,
                                     int64_t id_pad, void *out_d, int32_t out_bytes,
                                     dnatok_cuda_stream stream);

/* Algorithm 2's micro-batch size: min(emb_batch_cap, max(1, floor(
 * tokens_per_call / token_len))) rows. */
DNATOK_API dnatok_status dnatok_microbatch_rows(int64_t emb_batch_cap, int64_t tokens_per_call,
                                                int64_t token_len, int64_t *rows);

/*
 * Micro-batched feed on two streams (Sec. 2.2, "Pipelined streaming"): two
 * device buffers are used in turn, so the next micro-batch is written while
 * the consumer still works on the one before.  For each micro-batch of up to
 * rows_per_batch rows, dnatok_feed writes it into buf[i % 2] on
 * feed_stream; consumer_stream then waits for it and `consumer` is called
 * (on this host thread) to enqueue its work on consumer_stream; feed_stream
 * waits for that work before it reuses the buffer.  Each buffer holds
 * rows_per_batch x token_len elements of out_bytes.  ids and id_offsets
 * must be ready in consumer_stream's order (produced on it, or on a stream
 * it already waits for): feed_stream first waits for all work enqueued on
 * consumer_stream before the call.  Returns once everything is enqueued; a
 * nonzero return from `consumer` stops the loop with DNATOK_ERR_STATE.
 */
typedef int (*dnatok_feed_consumer)(void *user, int64_t row_begin, int64_t n_rows, void *batch_d,
                                    dnatok_cuda_stream consumer_stream);
DNATOK_API dnatok_status dnatok_feed_pipeline(const int32_t *ids_d, const int64_t *id_offsets_d,
                                              int64_t n_rows, int64_t token_len, int64_t id_pad,
                                              int32_t out_bytes, int64_t rows_per_batch,
                                              void *buf0_d, void *buf1_d,
                                              dnatok_cuda_stream feed_stream,
                                              dnatok_cuda_stream consumer_stream,
                                              dnatok_feed_consumer consumer, void *user);

/* --------------------------------------------------------------- shards */

/*
 * Byte-balanced contiguous record shards for encoding one batch with one
 * process per GPU.  Records are independent, so rank i encodes records
 * [bounds[i], bounds[i+1]) with no exchange on the data path; turning its
 * local id offsets into global ones needs only the exclusive scan of the
 * ranks' id counts (one integer per rank, done by the caller's collective).
 * bounds[0] = 0, bounds[world_size] = n_seq, and bounds[i] is the first
 * record that starts at or after i * n_bytes / world_size (records are never
 * split; one that spans a split point stays with the earlier rank).
 *   seq_offsets_host  n_seq + 1 non-decreasing int64 (HOST) with [0] = 0.
 *   bounds_out        world_size + 1 int64 (HOST).
 * Host only, no GPU work; DNATOK_ERR_ARG for bad arguments.
 */
DNATOK_API dnatok_status dnatok_shard_records(const int64_t *seq_offsets_host, int64_t n_seq,
                                              int32_t world_size, int64_t *bounds_out);

/* ------------------------------------------------------ no allocation */

/*
 * K-mer encode for callers that may not allocate device memory.  The paper
 * has no counterpart: this is a deployment form of dnatok_encode (RAW input,
 * mode DNATOK_KMER, the default base table) for code that runs where
 * cudaMalloc is off limits -- inside another library's memory pool, under a
 * framework whose allocator owns the whole device, or in a setting where an
 * allocation would synchronize the device.  It takes no handle and allocates
 * nothing: the look-back descriptors, counters and status word live in one
 * file-scope device array of fixed size, which every GPU that loads this
 * library holds until the process exits (about 0.5 MB).
 *
 *   k, bytes_d, seq_offsets_d, n_seq, ids_out_d, ids_capacity, id_offsets_d,
 *   offsets_capacity: as for dnatok_encode with a RAW k-mer handle (all
 *   DEVICE pointers owned by the caller).  ids_capacity must be at least
 *   min(n_bytes, (n_bytes + n_seq * (k - 1)) / k).
 *   totals_d: NULL or 2 int64 {number of ids, number of records}; both read
 *   -1 once the stream gets there if the kernel recorded a device-side error
 *   (such as malformed seq_offsets).
 *
 * n_bytes above DNATOK_NOALLOC_MAX_BYTES is rejected with
 * DNATOK_ERR_CAPACITY before anything is launched; bad arguments give
 * DNATOK_ERR_ARG, a failed CUDA call DNATOK_ERR_CUDA.
 *
 * The first call on a device (with that device current) looks up the
 * array's device address and caches it; make that first call before any
 * stream capture.  Every call clears the parts of the array it uses on
 * `stream` before launching.  All calls share the one array, so calls whose
 * work overlaps on the GPU (different streams, no ordering between them)
 * race: issue them on one stream or order them with events.
 */
#define DNATOK_NOALLOC_MAX_BYTES (1LL << 30)

DNATOK_API dnatok_status dnatok_encode_kmer_noalloc(int k, const uint8_t *bytes_d, int64_t n_bytes,
                                                    const int64_t *seq_offsets_d, int64_t n_seq,
                                                    int32_t *ids_out_d, int64_t ids_capacity,
                                                    int64_t *id_offsets_d,
                                                    int64_t offsets_capacity, int64_t *totals_d,
                                                    dnatok_cuda_stream stream);

/* -------------------------------------------------------------- launch */

/* Launch shape of the tokenization kernel: bytes per tile, threads per CTA,
 * resident CTAs per SM the grid is sized for (1..8), and tiles per chunk
 * (the unit of the cross-CTA look-back).  Supported (tile, threads, chunk):
 * (8192, 256, 8), (16384, 256, 4), (16384, 256, 8), (32768, 512, 4). */
typedef struct {
    int32_t tile_bytes;
    int32_t threads;
    int32_t ctas_per_sm;
    int32_t chunk_tiles;
} dnatok_launch_cfg;

DNATOK_API dnatok_status dnatok_get_launch(const dnatok_handle *h, dnatok_launch_cfg *cfg);
DNATOK_API dnatok_status dnatok_set_launch(dnatok_handle *h, const dnatok_launch_cfg *cfg);

/* ------------------------------------------------- graphs and autotuning */

/*
 * CUDA-graph capture (the batched form: one replay launches a whole batch,
 * or many encodes, with no per-call host work).  dnatok_graph_begin starts
 * capturing `stream` (a non-default stream, thread-local capture mode);
 * every dnatok_encode on it until dnatok_graph_end is recorded, not run.
 * Encodes recorded this way clear the look-back state they use inside the
 * graph, so replays are independent; all pointers are fixed in the graph
 * (refresh input bytes in place between replays).  Reserve workspace first
 * (dnatok_reserve): an encode that would have to allocate fails with
 * DNATOK_ERR_STATE under capture.  A handle must not run other work while
 * one of its graphs replays.  Not for the stream API (it waits on the host).
 */
typedef struct dnatok_graph dnatok_graph;
DNATOK_API dnatok_status dnatok_graph_begin(dnatok_handle *h, dnatok_cuda_stream stream);
DNATOK_API dnatok_status dnatok_graph_end(dnatok_handle *h, dnatok_cuda_stream stream,
                                          dnatok_graph **out);
DNATOK_API dnatok_status dnatok_graph_launch(dnatok_graph *g, dnatok_cuda_stream stream);
DNATOK_API void dnatok_graph_destroy(dnatok_graph *g);

/*
 * Autotuner: time every supported launch shape (tile bytes, threads, tiles
 * per chunk, resident CTAs per SM; for BPE handles the merge pass's segment
 * size; for k-mer handles whose RAW encodes take the direct path -- k >= 2,
 * dnatok_set_direct on, n_seq <= 65536 -- the direct kernel's slots per
 * step, ring depth and CTAs per SM) on this input -- `reps` timed runs each
 * after one warm-up, L2 flushed before each -- and keep the fastest on the
 * handle.  Arguments as
 * for dnatok_encode (device pointers; outputs are overwritten).  cache_path:
 * NULL or a text file; a line for this GPU, mode, k, format and input size
 * class (power of two) is reused without timing, and a new result is
 * appended.  best / best_ms (either may be NULL) receive the choice (for
 * BPE: {segment, halo, 0, 0}; for the direct path: {512 x slots per step,
 * 256 threads, CTAs per SM, ring steps}) and its mean time (-1 on a cache
 * hit).
 * Synchronizes; allocates a 192 MB scratch buffer while it runs.
 */
DNATOK_API dnatok_status dnatok_autotune(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                                         const int64_t *seq_offsets_d, int64_t n_seq,
                                         int32_t *ids_out_d, int64_t ids_capacity,
                                         int64_t *id_offsets_d, int64_t offsets_capacity,
                                         int32_t reps, const char *cache_path,
                                         dnatok_launch_cfg *best, float *best_ms);

/* RAW input through dnatok_encode first tries the direct path: when no byte
 * is below 0x21 (no separators), token positions follow from the record
 * lengths alone and the kernel needs no cross-tile scan; the general kernel
 * runs behind it only if the premise fails (same results either way).
 * enable = 0 sends every encode straight to the general kernel.  Default 1. */
DNATOK_API dnatok_status dnatok_set_direct(dnatok_handle *h, int32_t enable);

/* Which kernels finished the handle's last one-shot encode (dnatok_encode,
 * also inside dnatok_encode_host or dnatok_autotune): waits for `stream`,
 * then *out = 1 when the direct path produced every output, 0 when the
 * general kernel ran behind it (the direct path declined the input: a byte
 * below 0x21 in a record, a malformed seq_offsets, more FASTA records than
 * the direct plan takes, too few id offsets for the FASTA records), -1 when
 * the encode never tried the direct path (switched off, not eligible, or
 * no encode yet).  FASTA handles take the direct path for k-mers (k >= 2) of
 * 16-byte aligned text of 64 KiB up to 4 GiB: the text is first compacted on
 * the device to its sequence bytes and record starts.  DNATOK_KMER_TABLE
 * handles on RAW input take it straight from the bytes (window plan, count,
 * scan, expand), except under stream capture.  Not meaningful for an encode
 * recorded in a graph (its replays reset the switch). */
DNATOK_API dnatok_status dnatok_direct_ran(dnatok_handle *h, dnatok_cuda_stream stream,
                                           int32_t *out);

/* How long a look-back wait of the general kernel polls before it gives up
 * (each poll is followed by a sleep of up to about a microsecond): after
 * that many polls the kernel records a timeout and returns, and
 * dnatok_sync() reports DNATOK_ERR_TIMEOUT.  0 restores the default (about
 * four million polls).  Lower it to bound how long a stalled launch can
 * hold the GPU; tests lower it to see the timeout come back quickly. */
DNATOK_API dnatok_status dnatok_set_wait_limit(dnatok_handle *h, int64_t polls);

/* Kernel timing, for measurement: with enable != 0, every later one-shot
 * encode that runs the direct k-mer kernel (RAW input without separators,
 * k >= 2, not under stream capture) records two CUDA events on its stream,
 * right before and right after that kernel's launch; the kernel then waits
 * for the record plan to finish instead of starting under it.
 * dnatok_kernel_time_ms waits for `stream` and sets *ms to the time between
 * the two events of the last such encode on this handle, or to -1 when there
 * was none since timing was switched on.  0 switches it off (the default).
 * (No counterpart in the paper: a measurement aid.) */
DNATOK_API dnatok_status dnatok_set_kernel_timing(dnatok_handle *h, int32_t enable);
DNATOK_API dnatok_status dnatok_kernel_time_ms(dnatok_handle *h, dnatok_cuda_stream stream,
                                               float *ms);

/* Fault injection, for testing the bounded waits: the next launch of the
 * general kernel on this handle leaves look-back chunk `chunk` (chunks of
 * tiles_per_chunk x tile_bytes input bytes, counted from 0) unprocessed, so
 * the look-back of the chunk after it waits on a descriptor that is never
 * published and runs out (DNATOK_ERR_TIMEOUT from dnatok_sync; the
 * outputs of that launch are undefined).  -1 cancels.  Affects one launch.
 * (No counterpart in the paper.) */
DNATOK_API dnatok_status dnatok_inject_lookback_stall(dnatok_handle *h, int64_t chunk);

/* Shape of the direct k-mer kernel (RAW input without separators, k >= 2):
 * 512-byte slots per warp step ("bytes per thread": 16 per slot), warp
 * steps in its shared-memory ring ("pipeline depth": ring_steps - 1 steps in
 * flight per warp), and resident CTAs per SM the grid is sized for (0 = as
 * many as fit).  Supported: (slots, ring) in {(2, 4), (1, 8), (4, 2)},
 * ctas_per_sm 0..4; DNATOK_ERR_ARG otherwise.  Default (2, 4, 0).  Results
 * do not depend on the shape.  dnatok_autotune chooses it for handles that
 * take the direct path. */
DNATOK_API dnatok_status dnatok_set_direct_launch(dnatok_handle *h, int32_t slots_per_step,
                                                  int32_t ring_steps, int32_t ctas_per_sm);
/* out3 = {slots_per_step, ring_steps, ctas_per_sm}. */
DNATOK_API dnatok_status dnatok_get_direct_launch(const dnatok_handle *h, int32_t *out3);

/* BPE handles: symbols per segment of the merge pass (64..65536, a multiple
 * of 16, at least twice the longest token) and the halo each segment's pass
 * starts before it (0..seg_symbols, a multiple of 16).  A segment whose
 * halo pass does not agree with its left neighbour over the longest token's
 * length is recomputed exactly, so any halo gives the same ids; a short one
 * only costs time.  Defaults: 1024 and max(64, 4 x longest token). */
DNATOK_API dnatok_status dnatok_set_bpe_launch(dnatok_handle *h, int32_t seg_symbols, int32_t halo);
DNATOK_API dnatok_status dnatok_get_bpe_launch(const dnatok_handle *h, int32_t *seg_symbols,
                                               int32_t *halo);

/* BPE handles: statistics of the last encode on this handle, for tuning the
 * segment and halo sizes.  stats3[0] = symbols (kept bases and N-class bytes)
 * the merge pass ran over, stats3[1] = segments of seg_symbols symbols,
 * stats3[2] = segments whose halo pass did not agree with the neighbour to
 * their left and were recomputed exactly.  All zero before the first encode.
 * Synchronizes `stream` (the stream of that encode).  DNATOK_ERR_STATE on a
 * handle of another mode.  (Diagnostics of this library's own BPE method:
 * the paper defines no GPU BPE.) */
DNATOK_API dnatok_status dnatok_bpe_stats(dnatok_handle *h, int64_t *stats3,
                                          dnatok_cuda_stream stream);

/* ---- One long stream split into parts, one process (GPU) per part ----
 *
 * A part is a contiguous byte range of the stream (FASTA text, or RAW bytes
 * of one record), split anywhere: the streamed encode of Sec. 2.2 with its
 * chunks on different GPUs.  Each part's encode needs only a small state
 * from the bytes before it, the state that the host-streamed path
 * (dnatok_stream_*) carries from chunk to chunk: the scan element of the
 * encode at the part's start and the FASTA line state there.  The
 * protocol, for ranks 0..N-1 holding parts in stream order:
 *   1. every rank: dnatok_part_line_map of its part; exchange the maps; the
 *      line state at rank r's start is the stream start's state (0) mapped
 *      through the maps of ranks 0..r-1 in order;
 *   2. rank 0: dnatok_part_encode(before = NULL, last = (N == 1)), its real
 *      encode; ranks 1..N-2: dnatok_part_encode from an all-zero state in
 *      that line state, which gives the part's own state; exchange the
 *      states;
 *   3. rank r >= 1: its start state is rank 0's state combined
 *      (dnatok_part_combine, in order) with the states of ranks 1..r-1, with
 *      the line state of step 1; dnatok_part_encode(before = that, last =
 *      (r == N-1)).
 * Ranks exchange their part lengths with the maps: the first rank whose
 * part holds bytes plays rank 0 (ranks before it hold empty parts and write
 * nothing), so that the stream start merges with a header at its first byte
 * as in one encode.
 * Each rank's ids then start at its ids_out[0]: the part's ids are ids
 * [before.d, after.d) of the whole stream.  Its id_offsets[0 ..
 * after.nb - before.nb) are the offsets of records before.nb .. after.nb - 1
 * of the stream, as stream-wide id positions (the last part also writes the
 * final one).  Concatenated, the ranks' ids equal one encode of the stream.
 * Single-nucleotide and k-mer handles (not BPE, overlapping or table-driven
 * k-mers).
 */
typedef struct {
    int64_t nb;         /* record boundaries seen (the stream start counts) */
    int64_t h;          /* kept symbols before the first boundary */
    int64_t d;          /* ids completed */
    int64_t t;          /* kept symbols of the record still open */
    uint64_t codes;     /* its last min(t, k-1) symbols, 3 bits each, newest lowest;
                           their number in bits 58..61 */
    uint32_t line_state; /* FASTA: 0 at a line start, 1 in a header, 2 in sequence */
    uint32_t pad;
} dnatok_part_state;

/* The part's line-state map: bits 2s..2s+1 hold the state at its end when
 * it starts in state s (RAW handles: the identity, 0 | 1 << 2 | 2 << 4).
 * Reads the part's bytes on `stream` (DEVICE memory, any alignment) and
 * waits for the result. */
DNATOK_API dnatok_status dnatok_part_line_map(dnatok_handle *h, const uint8_t *bytes_d, int64_t n,
                                              int32_t *map_out, dnatok_cuda_stream stream);

/* Encode one part (DEVICE bytes, any alignment) from the state `before`
 * (host; NULL: the part starts the stream) and write the state at its end
 * to *after (host).  last != 0: the part ends the stream (the open record
 * is closed).  A `before` with nb = 0 (all zero but the line state) asks
 * for the part's own state, the one that dnatok_part_combine appends to the
 * state before it: the outputs are then scratch (two runs of the encode for
 * k-mers, one for single nucleotides).  ids_out_d: ids_capacity >= n + 1;
 * id_offsets_d: offsets_capacity >= 1 entries, those past it not written.
 * Waits for `stream`; device errors come back as from dnatok_sync.
 * DNATOK_ERR_STATE for BPE, overlapping or table-driven handles, or while a
 * stream is open on h. */
DNATOK_API dnatok_status dnatok_part_encode(dnatok_handle *h, const uint8_t *bytes_d, int64_t n,
                                            const dnatok_part_state *before, int32_t last,
                                            int32_t *ids_out_d, int64_t ids_capacity,
                                            int64_t *id_offsets_d, int64_t offsets_capacity,
                                            dnatok_part_state *after, dnatok_cuda_stream stream);

/* out = the state after a part with state b that follows a stretch of the
 * stream with state a, for k-mers of k (1 for single nucleotides).  Host
 * only (no device work).  The line state is b's. */
DNATOK_API dnatok_status dnatok_part_combine(int32_t k, const dnatok_part_state *a,
                                             const dnatok_part_state *b, dnatok_part_state *out);

#ifdef __cplusplus
}
#endif
#endif /* DNATOK_H */
