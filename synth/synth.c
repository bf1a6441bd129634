/*
 * synth.c -- seeded synthetic DNA byte generators.
 *
 * These routines only produce INPUT bytes (sequences, FASTA text, request
 * payloads).  They contain no tokenizer arithmetic: no byte classes, no IDs,
 * no k-mer or BPE logic.  Both the CPU oracle tests and the CUDA-path tests
 * feed on the same generated bytes.
 *
 * Random numbers: splitmix64 (Steele, Lea & Flood 2014, "Fast splittable
 * pseudorandom number generators"), one independent counter stream per
 * (seed, sequence index), so output does not depend on the thread count.
 *
 * Integer-only sampling: probabilities arrive as 32-bit thresholds and
 * log-uniform stretch lengths as a quantile table, both computed by the
 * Python side.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream_seed(uint64_t seed, uint64_t stream, uint64_t salt) {
    uint64_t s = seed * 0xD1B54A32D192ED03ULL ^ (stream + 1) * 0x9E3779B97F4A7C15ULL ^ salt;
    (void)sm64_next(&s);
    return s;
}

static const uint8_t ACGT[4] = {'A', 'C', 'G', 'T'};

/* Order-3 Markov chain over ACGT.  cdf holds, for each of the 64 contexts
 * (16*b[-3] + 4*b[-2] + b[-1]), three cumulative 32-bit thresholds. */
static void fill_markov(uint8_t *out, int64_t n, const uint32_t *cdf, uint64_t *rng) {
    uint32_t ctx = (uint32_t)(sm64_next(rng) & 63u);
    int64_t i = 0;
    while (i < n) {
        uint64_t r = sm64_next(rng);
        for (int h = 0; h < 2 && i < n; ++h, ++i) {
            uint32_t u = (uint32_t)(r >> (32 * h));
            const uint32_t *c = cdf + 3 * ctx;
            uint32_t b = (u >= c[0]) + (u >= c[1]) + (u >= c[2]);
            out[i] = ACGT[b];
            ctx = ((ctx << 2) | b) & 63u;
        }
    }
}

static void fill_iid(uint8_t *out, int64_t n, uint64_t *rng) {
    int64_t i = 0;
    while (i < n) {
        uint64_t r = sm64_next(rng);
        for (int h = 0; h < 32 && i < n; ++h, ++i) out[i] = ACGT[(r >> (2 * h)) & 3u];
    }
}

/* Runs of 'N': a run starts at a position with probability start_p32/2^32,
 * its length uniform in [lo, hi]. */
static void add_nruns(uint8_t *out, int64_t n, uint32_t start_p32, int lo, int hi, uint64_t *rng) {
    if (start_p32 == 0) return;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t r = sm64_next(rng);
        if ((uint32_t)r < start_p32) {
            int64_t len = lo + (int64_t)((r >> 32) % (uint64_t)(hi - lo + 1));
            for (int64_t j = 0; j < len && i < n; ++j, ++i) out[i] = 'N';
        }
    }
}

/* Lowercase (soft-masked) stretches: start probability start_p32/2^32, length
 * drawn from a 4096-entry quantile table. */
static void add_lower_stretches(uint8_t *out, int64_t n, uint32_t start_p32,
                                const int32_t *len_table, uint64_t *rng) {
    if (start_p32 == 0) return;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t r = sm64_next(rng);
        if ((uint32_t)r < start_p32) {
            int64_t len = len_table[(r >> 32) & 4095u];
            for (int64_t j = 0; j < len && i < n; ++j, ++i)
                if (out[i] >= 'A' && out[i] <= 'Z') out[i] = (uint8_t)(out[i] + 32);
        }
    }
}

/* Independent per-byte lowercase with probability p32/2^32. */
static void lower_iid(uint8_t *out, int64_t n, uint32_t p32, uint64_t *rng) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u = (uint32_t)sm64_next(rng);
        if (u < p32 && out[i] >= 'A' && out[i] <= 'Z') out[i] = (uint8_t)(out[i] + 32);
    }
}

/* ---------------------------------------------------------------- public */

void synth_iid_sequence(uint8_t *out, int64_t n, uint32_t nrun_p32, int nrun_lo, int nrun_hi,
                        uint32_t lower_p32, uint64_t seed) {
    uint64_t rng = stream_seed(seed, 0, 1);
    fill_iid(out, n, &rng);
    uint64_t rn = stream_seed(seed, 0, 2);
    add_nruns(out, n, nrun_p32, nrun_lo, nrun_hi, &rn);
    uint64_t rl = stream_seed(seed, 0, 3);
    lower_iid(out, n, lower_p32, &rl);
}

typedef struct {
    uint8_t *out;
    const int64_t *offsets;
    int64_t n_seq;
    const uint32_t *cdf;
    uint32_t nrun_p32;
    int nrun_lo, nrun_hi;
    uint32_t lower_p32;
    const int32_t *len_table;
    uint64_t seed;
    int64_t next, end;  /* records [next, end) are still to be written */
    int64_t base;       /* byte offset of out[0] in the whole batch */
    pthread_mutex_t lock;
} batch_job;

static void batch_one(batch_job *J, int64_t s) {
    uint8_t *p = J->out + (J->offsets[s] - J->base);
    int64_t n = J->offsets[s + 1] - J->offsets[s];
    uint64_t rm = stream_seed(J->seed, (uint64_t)s, 11);
    fill_markov(p, n, J->cdf, &rm);
    uint64_t rn = stream_seed(J->seed, (uint64_t)s, 12);
    add_nruns(p, n, J->nrun_p32, J->nrun_lo, J->nrun_hi, &rn);
    uint64_t rl = stream_seed(J->seed, (uint64_t)s, 13);
    add_lower_stretches(p, n, J->lower_p32, J->len_table, &rl);
}

static void *batch_worker(void *arg) {
    batch_job *J = (batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t s = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (s >= J->end) break;
        batch_one(J, s);
    }
    return NULL;
}

/* Fill Markov sequences [first, last) of a batch laid out back to back at
 * offsets[0..n_seq]; out holds bytes offsets[first] .. offsets[last]. */
void synth_markov_batch(uint8_t *out, const int64_t *offsets, int64_t n_seq, const uint32_t *cdf,
                        uint32_t nrun_p32, int nrun_lo, int nrun_hi, uint32_t lower_p32,
                        const int32_t *len_table, uint64_t seed, int n_threads, int64_t first,
                        int64_t last) {
    batch_job J;
    J.out = out; J.offsets = offsets; J.n_seq = n_seq; J.cdf = cdf;
    J.nrun_p32 = nrun_p32; J.nrun_lo = nrun_lo; J.nrun_hi = nrun_hi;
    J.lower_p32 = lower_p32; J.len_table = len_table; J.seed = seed;
    if (first < 0) first = 0;
    if (last > n_seq) last = n_seq;
    J.next = first; J.end = last;
    J.base = (first < n_seq) ? offsets[first] : 0;
    pthread_mutex_init(&J.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, batch_worker, &J);
    batch_worker(&J);
    for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.lock);
}

/* ------------------------------------------------------------ FASTA text */

typedef struct {
    uint8_t *out;
    int64_t n_total;
    int64_t n_rec;
    const int64_t *rec_off;   /* byte offset of each record's '>' */
    const int32_t *hdr_len;   /* header characters including '>' (newline excluded) */
    const int32_t *wrap;      /* sequence line width */
    const int64_t *seq_len;   /* bases in the record */
    const uint32_t *cdf;
    uint32_t nrun_p32;
    int nrun_lo, nrun_hi;
    uint32_t lower_p32;
    const int32_t *len_table;
    uint64_t seed;
    int64_t next, end;  /* records [next, end) are still to be written */
    int64_t base;       /* byte offset of out[0] in the whole stream */
    pthread_mutex_t lock;
} fasta_job;

static void fasta_one(fasta_job *J, int64_t r, uint8_t *scratch) {
    int64_t off = J->rec_off[r];
    int64_t end = (r + 1 < J->n_rec) ? J->rec_off[r + 1] : J->n_total;
    uint8_t *p = J->out + (off - J->base);
    int64_t room = end - off;
    uint64_t rh = stream_seed(J->seed, (uint64_t)r, 21);
    int64_t w = 0;
    if (w < room) p[w++] = '>';
    for (int32_t c = 1; c < J->hdr_len[r] && w < room; ++c) {
        uint64_t u = sm64_next(&rh);
        p[w++] = (uint8_t)(32 + (u % 95u)); /* printable ASCII 32..126 */
    }
    if (w < room) p[w++] = '\n';
    int64_t n = J->seq_len[r];
    uint64_t rm = stream_seed(J->seed, (uint64_t)r, 22);
    fill_markov(scratch, n, J->cdf, &rm);
    uint64_t rn = stream_seed(J->seed, (uint64_t)r, 23);
    add_nruns(scratch, n, J->nrun_p32, J->nrun_lo, J->nrun_hi, &rn);
    uint64_t rl = stream_seed(J->seed, (uint64_t)r, 24);
    add_lower_stretches(scratch, n, J->lower_p32, J->len_table, &rl);
    int64_t col = 0;
    for (int64_t i = 0; i < n && w < room; ++i) {
        p[w++] = scratch[i];
        if (++col == J->wrap[r] && w < room) { p[w++] = '\n'; col = 0; }
    }
    if (col != 0 && w < room) p[w++] = '\n';
    while (w < room) p[w++] = '\n'; /* only if the layout over-allocated */
}

static void *fasta_worker(void *arg) {
    fasta_job *J = (fasta_job *)arg;
    int64_t cap = 0;
    uint8_t *scratch = NULL;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t r = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (r >= J->end) break;
        if (J->seq_len[r] > cap) {
            free(scratch);
            cap = J->seq_len[r];
            scratch = (uint8_t *)malloc((size_t)cap + 1);
            if (!scratch) { cap = 0; continue; }
        }
        fasta_one(J, r, scratch);
    }
    free(scratch);
    return NULL;
}

/* Write n_rec FASTA records at the byte offsets rec_off (computed by the
 * caller so that each record occupies exactly its header line plus its
 * wrapped sequence lines); only records [first, last) are written, out
 * holding bytes rec_off[first] onwards. */
void synth_fasta(uint8_t *out, int64_t n_total, int64_t n_rec, const int64_t *rec_off,
                 const int32_t *hdr_len, const int32_t *wrap, const int64_t *seq_len,
                 const uint32_t *cdf, uint32_t nrun_p32, int nrun_lo, int nrun_hi,
                 uint32_t lower_p32, const int32_t *len_table, uint64_t seed, int n_threads,
                 int64_t first, int64_t last) {
    fasta_job J;
    J.out = out; J.n_total = n_total; J.n_rec = n_rec; J.rec_off = rec_off;
    J.hdr_len = hdr_len; J.wrap = wrap; J.seq_len = seq_len; J.cdf = cdf;
    J.nrun_p32 = nrun_p32; J.nrun_lo = nrun_lo; J.nrun_hi = nrun_hi;
    J.lower_p32 = lower_p32; J.len_table = len_table; J.seed = seed;
    if (first < 0) first = 0;
    if (last > n_rec) last = n_rec;
    J.next = first; J.end = last;
    J.base = (first < n_rec) ? rec_off[first] : 0;
    pthread_mutex_init(&J.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, fasta_worker, &J);
    fasta_worker(&J);
    for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.lock);
}

/* Uniformly random bytes (any value 0..255), for fuzzing byte classification. */
void synth_random_bytes(uint8_t *out, int64_t n, uint64_t seed) {
    uint64_t rng = stream_seed(seed, 0, 31);
    int64_t i = 0;
    while (i < n) {
        uint64_t r = sm64_next(&rng);
        for (int h = 0; h < 8 && i < n; ++h, ++i) out[i] = (uint8_t)(r >> (8 * h));
    }
}
