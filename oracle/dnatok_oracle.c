/*
 * dnatok_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of what the DNA byte ->
 * token-ID path computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library; the two are written apart and
 * compared on the same generated bytes.
 *
 * What it follows (Niktab & Patel, "DNATokenizer: A GPU-First
 * Byte-to-Identifier Tokenizer", arXiv 2601.05531):
 *   - the 256-entry byte -> identifier table and its fixed DNA fallback
 *     (Algorithm 1, DiscoverIDsPath), applied as ascii_lut[Bytes]
 *     (Sec. 2.2 "Bytes path", Algorithm 2);
 *   - non-overlapping k-mers: tokens of k bases sharing no bases, which
 *     shrink the length by k (Sec. 1.1, Table 1), built from base digits
 *     (MapKmer in Algorithm 2) -- here the closed form
 *     id = sum_i 4^(k-1-i) * code(b_i);
 *   - BPE with a fixed, rank-ordered merge table whose segmentation and
 *     IDs must match the source tokenizer (Sec. 1.1, Sec. 4.3);
 *   - overlapping k-mers (a window at every position): each run of k
 *     consecutive bases is one token, so neighbours overlap in all but one
 *     base, and an input of L bases gives
 *     L-k+1 tokens (Sec. 1.1, Table 1).
 *
 * Readings where the paper is silent (each one is a test in tests/):
 *   C1  case-insensitive: a/c/g/t/n behave like A/C/G/T/N (Algorithm 1).
 *   C2  every byte that is not A/C/G/T (either case) or one of the four
 *       separators below is N-class (IUPAC codes, digits, bytes >= 128, NUL).
 *   C3  '\n', '\r', ' ', '\t' are dropped; they emit nothing and do not move
 *       the k-mer frame; a BPE word continues across them.
 *   C4  FASTA: a line whose first byte is '>' is a header; it is dropped up to
 *       and including its '\n' and starts a new record.  Bytes before the
 *       first header form a record only when byte 0 is not '>'.
 *   C5  single-nucleotide default table: A0 C1 G2 T3, every N-class byte 4,
 *       separators dropped (-1).  Any user table of 256 ids (-1 = drop) is
 *       accepted, e.g. the paper's fallback A1 C2 G3 T4 N0.
 *   C6  k-mers: frame per record over kept bases; a token with any N-class
 *       base is UNK = 4^k; a tail of L mod k > 0 bases emits one UNK.
 *   C7  BPE: base ids A0 C1 G2 T3, merge rank r -> id 4+r, N_ID = 4+M.
 *       Greedy: repeatedly merge the adjacent pair of lowest rank, leftmost
 *       first, until no adjacent pair is in the table.
 *   C8  BPE words are maximal runs of bases inside one record; an N-class
 *       byte ends the word and emits N_ID.
 *   C9  trainer: overlapping pair counts, maximum count wins, ties go to the
 *       smallest (left, right); stop when the best count is below 2; each
 *       merge is applied left to right without overlap.
 *   C10 ids are int32, record offsets int64.
 *   C15 overlapping k-mers: per record over kept bases (as C6), one token for
 *       every start j <= L - k with the C6 ids (any N-class base: UNK = 4^k);
 *       a record with L < k bases has no token.
 *   C16 table-driven k-mers (Algorithm 1 builds kmer_lut[0..5^k-1] and a
 *       byte -> base-5 digit table; Algorithm 2 applies MapKmer): digits A0
 *       C1 G2 T3, every N-class byte 4 (C1-C3); the record's kept symbols are
 *       cut into windows of k from its start (as C6); a whole window with
 *       index sum_i 5^(k-1-i) d_i emits kmer_lut[index] when that entry is
 *       >= 0, else each of its k symbols as base_ids[d]; a tail of L mod k
 *       symbols emits base_ids[d] for each one.  1 <= k <= 10.
 *   C17 decode (Sec. 4, "Decode Operations"; a reverse id -> text lookup):
 *       single-nucleotide ids through the inverse of the handle's 256-entry
 *       table -- for id v the first byte b in the order "ACGTN", then 'A'..'Z',
 *       'a'..'z', then 0..255, with lut[b] == v; table-driven k-mer ids
 *       through the smallest index with kmer_lut[index] == v (its k digits
 *       written as "ACGTN"), else the smallest digit with base_ids[d] == v.
 *       An id with no inverse is an error.
 *   C18 reverse complement (Sec. 4, "Integration with Data Augmentation"):
 *       per record, out[s + e - 1 - i] = comp(in[i]); comp swaps A/T, C/G,
 *       R/Y, K/M, B/V, D/H in either case, keeps S W N and every other byte.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_CHAR = 0, OR_KMER = 1, OR_BPE = 2, OR_KMER_OVL = 3, OR_KMER_TABLE = 4 };
enum { OR_RAW = 0, OR_FASTA = 1 };
enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_CAPACITY = -3, OR_ERR_NOMEM = -8 };

/* ------------------------------------------------------------ byte classes */

enum { K_BASE = 0, K_NCLASS = 1, K_DROP = 2 };

/* C1-C3: classify one byte; for bases also return the 2-bit code. */
static int classify(uint8_t b, int *code) {
    switch (b) {
    case 'A': case 'a': *code = 0; return K_BASE;
    case 'C': case 'c': *code = 1; return K_BASE;
    case 'G': case 'g': *code = 2; return K_BASE;
    case 'T': case 't': *code = 3; return K_BASE;
    case '\n': case '\r': case ' ': case '\t': return K_DROP;
    default: return K_NCLASS;
    }
}

/* C5: the default single-nucleotide table. */
void oracle_default_lut(int32_t *lut) {
    for (int b = 0; b < 256; ++b) {
        int code = 0;
        int k = classify((uint8_t)b, &code);
        lut[b] = (k == K_BASE) ? code : (k == K_DROP ? -1 : 4);
    }
}

/* ------------------------------------------------------------ record split */

/* RAW: records are [seq_offsets[r], seq_offsets[r+1]).  FASTA (C4): walk the
 * lines; a '>' at a line start opens a record and the whole line is marked as
 * header.  Returns the number of records; rec_start gets n_rec + 1 entries
 * (the last one is n). */
static int64_t split_records(int fmt, const uint8_t *bytes, int64_t n, const int64_t *seq_offsets,
                             int64_t n_seq, int64_t **rec_start_out, uint8_t **in_header_out) {
    uint8_t *hdr = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *rs = NULL;
    int64_t n_rec = 0;
    if (!hdr) return -1;
    if (fmt == OR_RAW) {
        rs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_seq + 1));
        if (!rs) { free(hdr); return -1; }
        for (int64_t r = 0; r <= n_seq; ++r) rs[r] = seq_offsets[r];
        n_rec = n_seq;
    } else {
        int64_t cap = 16;
        rs = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        if (!rs) { free(hdr); return -1; }
        if (n > 0 && bytes[0] != '>') rs[n_rec++] = 0;
        int line_start = 1, in_header = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (line_start) {
                in_header = (bytes[i] == '>');
                if (in_header) {
                    if (n_rec + 2 > cap) {
                        cap *= 2;
                        int64_t *t = (int64_t *)realloc(rs, sizeof(int64_t) * (size_t)cap);
                        if (!t) { free(rs); free(hdr); return -1; }
                        rs = t;
                    }
                    rs[n_rec++] = i;
                }
            }
            hdr[i] = (uint8_t)in_header;
            line_start = (bytes[i] == '\n');
        }
        rs[n_rec] = n;
    }
    *rec_start_out = rs;
    *in_header_out = hdr;
    return n_rec;
}

/* ----------------------------------------------------------------- BPE */

typedef struct { int32_t left, right, rank; } pair_rank;

static int cmp_pair(const void *a, const void *b) {
    const pair_rank *x = (const pair_rank *)a, *y = (const pair_rank *)b;
    if (x->left != y->left) return x->left < y->left ? -1 : 1;
    if (x->right != y->right) return x->right < y->right ? -1 : 1;
    return 0;
}

typedef struct { pair_rank *p; int32_t m; } rank_table;

static int build_rank_table(const int32_t *merges, int32_t m, rank_table *t) {
    t->m = m;
    t->p = (pair_rank *)malloc(sizeof(pair_rank) * (size_t)(m > 0 ? m : 1));
    if (!t->p) return -1;
    for (int32_t r = 0; r < m; ++r) {
        t->p[r].left = merges[2 * r];
        t->p[r].right = merges[2 * r + 1];
        t->p[r].rank = r;
    }
    qsort(t->p, (size_t)m, sizeof(pair_rank), cmp_pair);
    return 0;
}

/* Rank of the pair (a, b) in the merge table, or -1. */
static int32_t rank_of(const rank_table *t, int32_t a, int32_t b) {
    pair_rank key = {a, b, 0};
    const pair_rank *hit = (const pair_rank *)bsearch(&key, t->p, (size_t)t->m,
                                                      sizeof(pair_rank), cmp_pair);
    return hit ? hit->rank : -1;
}

typedef struct { int32_t rank; int64_t pos; } heap_ent;

static int heap_less(heap_ent a, heap_ent b) {
    return a.rank < b.rank || (a.rank == b.rank && a.pos < b.pos);
}

typedef struct { heap_ent *a; int64_t n, cap; } heap_t;

static int heap_push(heap_t *h, int32_t rank, int64_t pos) {
    if (h->n == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 64;
        heap_ent *t = (heap_ent *)realloc(h->a, sizeof(heap_ent) * (size_t)nc);
        if (!t) return -1;
        h->a = t; h->cap = nc;
    }
    int64_t i = h->n++;
    heap_ent e = {rank, pos};
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!heap_less(e, h->a[p])) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i] = e;
    return 0;
}

static heap_ent heap_pop(heap_t *h) {
    heap_ent top = h->a[0];
    heap_ent last = h->a[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        heap_ent best = last;
        if (l < h->n && heap_less(h->a[l], best)) { best = h->a[l]; s = l; }
        if (r < h->n && heap_less(h->a[r], best)) { best = h->a[r]; s = r; }
        if (s == i) break;
        h->a[i] = h->a[s];
        i = s;
    }
    if (h->n > 0) h->a[i] = last;
    return top;
}

/* C7: greedy BPE on one word of base codes (0..3).  A doubly linked list of
 * symbols and a min-heap of (rank, position) with lazy invalidation: an entry
 * is used only if its left symbol is alive, has a right neighbour, and that
 * pair still has the entry's rank.  Writes the tokens to out, returns count. */
static int64_t bpe_word(const rank_table *t, const int32_t *codes, int64_t L, int32_t *out) {
    if (L <= 0) return 0;
    int32_t *tok = (int32_t *)malloc(sizeof(int32_t) * (size_t)L);
    int64_t *nxt = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    int64_t *prv = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    uint8_t *alive = (uint8_t *)malloc((size_t)L);
    heap_t h = {NULL, 0, 0};
    int64_t n_out = -1;
    if (!tok || !nxt || !prv || !alive) goto done;
    for (int64_t i = 0; i < L; ++i) {
        tok[i] = codes[i];
        nxt[i] = (i + 1 < L) ? i + 1 : -1;
        prv[i] = i - 1;
        alive[i] = 1;
    }
    for (int64_t i = 0; i + 1 < L; ++i) {
        int32_t r = rank_of(t, tok[i], tok[i + 1]);
        if (r >= 0 && heap_push(&h, r, i)) goto done;
    }
    while (h.n > 0) {
        heap_ent e = heap_pop(&h);
        int64_t i = e.pos;
        if (!alive[i]) continue;
        int64_t j = nxt[i];
        if (j < 0 || rank_of(t, tok[i], tok[j]) != e.rank) continue;
        tok[i] = 4 + e.rank;
        alive[j] = 0;
        nxt[i] = nxt[j];
        if (nxt[j] >= 0) prv[nxt[j]] = i;
        if (prv[i] >= 0) {
            int32_t r = rank_of(t, tok[prv[i]], tok[i]);
            if (r >= 0 && heap_push(&h, r, prv[i])) goto done;
        }
        if (nxt[i] >= 0) {
            int32_t r = rank_of(t, tok[i], tok[nxt[i]]);
            if (r >= 0 && heap_push(&h, r, i)) goto done;
        }
    }
    n_out = 0;
    for (int64_t i = 0; i >= 0; i = nxt[i]) out[n_out++] = tok[i];
done:
    free(tok); free(nxt); free(prv); free(alive); free(h.a);
    return n_out;
}

/* Greedy BPE of one word given as base codes; exported for the tests. */
int64_t oracle_bpe_word(const int32_t *merges, int32_t n_merges, const int32_t *codes, int64_t L,
                        int32_t *out) {
    rank_table t;
    if (build_rank_table(merges, n_merges, &t)) return OR_ERR_NOMEM;
    int64_t n = bpe_word(&t, codes, L, out);
    free(t.p);
    return n < 0 ? OR_ERR_NOMEM : n;
}

/* -------------------------------------------------------------- encode */

/*
 * Encode a byte stream.  mode: 0 single-nucleotide, 1 k-mer, 2 BPE,
 * 3 overlapping (stride-1) k-mer.
 * fmt: 0 RAW (records given by seq_offsets[0..n_seq]), 1 FASTA (records
 * found from header lines).  lut: 256 ids for mode 0 (NULL = default C5).
 * Outputs: ids (capacity ids_cap), offsets (capacity offs_cap >= n_rec + 1),
 * *n_ids, *n_rec.  Returns 0, or a negative code.
 */
int oracle_encode(int mode, int k, const int32_t *lut_in, const int32_t *merges,
                  int32_t n_merges, int fmt, const uint8_t *bytes, int64_t n,
                  const int64_t *seq_offsets, int64_t n_seq, int32_t *ids, int64_t ids_cap,
                  int64_t *offsets, int64_t offs_cap, int64_t *n_ids_out, int64_t *n_rec_out) {
    if (mode < 0 || mode > 3 || fmt < 0 || fmt > 1 || n < 0) return OR_ERR_ARG;
    if ((mode == OR_KMER || mode == OR_KMER_OVL) && (k < 1 || k > 15)) return OR_ERR_ARG;
    if (fmt == OR_RAW) {
        if (n_seq < 0 || !seq_offsets || seq_offsets[0] != 0 || seq_offsets[n_seq] != n)
            return OR_ERR_ARG;
        for (int64_t r = 0; r < n_seq; ++r)
            if (seq_offsets[r + 1] < seq_offsets[r]) return OR_ERR_ARG;
    }
    int32_t lut[256];
    if (mode == OR_CHAR) {
        if (lut_in) memcpy(lut, lut_in, sizeof(lut));
        else oracle_default_lut(lut);
    }
    rank_table rt = {NULL, 0};
    if (mode == OR_BPE && build_rank_table(merges, n_merges, &rt)) return OR_ERR_NOMEM;

    int64_t *rs = NULL;
    uint8_t *hdr = NULL;
    int64_t n_rec = split_records(fmt, bytes, n, seq_offsets, n_seq, &rs, &hdr);
    if (n_rec < 0) { free(rt.p); return OR_ERR_NOMEM; }

    int32_t *sym = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *word_out = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int status = OR_OK;
    int64_t w = 0;
    if (!sym || !word_out) { status = OR_ERR_NOMEM; goto out; }
    if (n_rec + 1 > offs_cap) { status = OR_ERR_CAPACITY; goto out; }

    for (int64_t r = 0; r < n_rec; ++r) {
        offsets[r] = w;
        /* the record's kept symbols, in order */
        int64_t L = 0;
        for (int64_t i = rs[r]; i < rs[r + 1]; ++i) {
            if (hdr[i]) continue;
            if (mode == OR_CHAR) {
                if (lut[bytes[i]] >= 0) sym[L++] = lut[bytes[i]];
            } else {
                int code = 0, c = classify(bytes[i], &code);
                if (c == K_BASE) sym[L++] = code;
                else if (c == K_NCLASS) sym[L++] = -1; /* N-class marker */
            }
        }
        if (mode == OR_CHAR) {
            if (w + L > ids_cap) { status = OR_ERR_CAPACITY; goto out; }
            for (int64_t j = 0; j < L; ++j) ids[w++] = sym[j];
        } else if (mode == OR_KMER) {
            int64_t unk = (int64_t)1 << (2 * k);
            int64_t n_tok = (L + k - 1) / k;
            if (w + n_tok > ids_cap) { status = OR_ERR_CAPACITY; goto out; }
            for (int64_t t = 0; t < n_tok; ++t) {
                int64_t id = 0;
                if ((t + 1) * k > L) {
                    id = unk; /* C6 tail */
                } else {
                    for (int i = 0; i < k; ++i) {
                        int32_t c = sym[t * k + i];
                        if (c < 0) { id = unk; break; }
                        id = id * 4 + c;
                    }
                }
                ids[w++] = (int32_t)id;
            }
        } else if (mode == OR_KMER_OVL) {
            /* C15: a token at every start j with j + k <= L */
            int64_t unk = (int64_t)1 << (2 * k);
            int64_t n_tok = L >= k ? L - k + 1 : 0;
            if (w + n_tok > ids_cap) { status = OR_ERR_CAPACITY; goto out; }
            for (int64_t j = 0; j < n_tok; ++j) {
                int64_t id = 0;
                for (int i = 0; i < k; ++i) {
                    int32_t c = sym[j + i];
                    if (c < 0) { id = unk; break; }
                    id = id * 4 + c;
                }
                ids[w++] = (int32_t)id;
            }
        } else {
            int32_t n_id = 4 + n_merges;
            int64_t j = 0;
            while (j < L) {
                if (sym[j] < 0) {
                    if (w + 1 > ids_cap) { status = OR_ERR_CAPACITY; goto out; }
                    ids[w++] = n_id;
                    ++j;
                    continue;
                }
                int64_t e = j;
                while (e < L && sym[e] >= 0) ++e;
                int64_t m = bpe_word(&rt, sym + j, e - j, word_out);
                if (m < 0) { status = OR_ERR_NOMEM; goto out; }
                if (w + m > ids_cap) { status = OR_ERR_CAPACITY; goto out; }
                for (int64_t q = 0; q < m; ++q) ids[w++] = word_out[q];
                j = e;
            }
        }
    }
    offsets[n_rec] = w;
    *n_ids_out = w;
    *n_rec_out = n_rec;
out:
    free(sym); free(word_out); free(rs); free(hdr); free(rt.p);
    return status;
}

/* -------------------------------------------------------------- trainer */

/* C9: train up to n_merges merges on one word of base codes (0..3).
 * Returns the number of merges written to merges_out (2 ints each). */
int32_t oracle_bpe_train(const uint8_t *codes, int64_t n, int32_t n_merges, int32_t *merges_out) {
    int64_t V = 4 + (int64_t)n_merges;
    int32_t *seq = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *count = (int32_t *)calloc((size_t)(V * V), sizeof(int32_t));
    int64_t *touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 1 ? n : 1));
    int32_t r = 0;
    if (!seq || !count || !touched) { r = OR_ERR_NOMEM; goto done; }
    for (int64_t i = 0; i < n; ++i) seq[i] = codes[i];
    int64_t len = n;
    for (r = 0; r < n_merges; ++r) {
        int64_t n_touched = 0;
        for (int64_t i = 0; i + 1 < len; ++i) {
            int64_t key = (int64_t)seq[i] * V + seq[i + 1];
            if (count[key]++ == 0) touched[n_touched++] = key;
        }
        int64_t best = -1;
        int32_t best_count = 0;
        for (int64_t q = 0; q < n_touched; ++q) {
            int64_t key = touched[q];
            if (count[key] > best_count || (count[key] == best_count && key < best)) {
                best = key;
                best_count = count[key];
            }
            count[key] = 0;
        }
        if (best_count < 2) break;
        int32_t L = (int32_t)(best / V), R = (int32_t)(best % V);
        merges_out[2 * r] = L;
        merges_out[2 * r + 1] = R;
        int64_t wr = 0;
        for (int64_t i = 0; i < len;) {
            if (i + 1 < len && seq[i] == L && seq[i + 1] == R) {
                seq[wr++] = 4 + r;
                i += 2;
            } else {
                seq[wr++] = seq[i++];
            }
        }
        len = wr;
    }
done:
    free(seq); free(count); free(touched);
    return r;
}

/* ------------------------------------------------- table-driven k-mers */

/* C16: tokens of every record through kmer_lut (5^k entries, -1 = no entry)
 * and base_ids (5 entries for the digits A C G T N).  Arguments and results
 * as oracle_encode. */
int oracle_encode_ktab(int k, const int32_t *kmer_lut, const int32_t *base_ids, int fmt,
                       const uint8_t *bytes, int64_t n, const int64_t *seq_offsets,
                       int64_t n_seq, int32_t *ids, int64_t ids_cap, int64_t *offsets,
                       int64_t offs_cap, int64_t *n_ids_out, int64_t *n_rec_out) {
    if (k < 1 || k > 10 || !kmer_lut || !base_ids || fmt < 0 || fmt > 1 || n < 0)
        return OR_ERR_ARG;
    if (fmt == OR_RAW) {
        if (n_seq < 0 || !seq_offsets || seq_offsets[0] != 0 || seq_offsets[n_seq] != n)
            return OR_ERR_ARG;
        for (int64_t r = 0; r < n_seq; ++r)
            if (seq_offsets[r + 1] < seq_offsets[r]) return OR_ERR_ARG;
    }
    int64_t *rs = NULL;
    uint8_t *hdr = NULL;
    int64_t n_rec = split_records(fmt, bytes, n, seq_offsets, n_seq, &rs, &hdr);
    if (n_rec < 0) return OR_ERR_NOMEM;
    int32_t *digit = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int status = OR_OK;
    int64_t w = 0;
    if (!digit) { status = OR_ERR_NOMEM; goto out; }
    if (n_rec + 1 > offs_cap) { status = OR_ERR_CAPACITY; goto out; }
    for (int64_t r = 0; r < n_rec; ++r) {
        offsets[r] = w;
        int64_t L = 0;
        for (int64_t i = rs[r]; i < rs[r + 1]; ++i) {
            if (hdr[i]) continue;
            int code = 0, c = classify(bytes[i], &code);
            if (c == K_BASE) digit[L++] = code;
            else if (c == K_NCLASS) digit[L++] = 4;
        }
        int64_t t = 0;
        for (; t + k <= L; t += k) {  /* whole windows */
            int64_t index = 0;
            for (int i = 0; i < k; ++i) index = index * 5 + digit[t + i];
            if (kmer_lut[index] >= 0) {
                if (w + 1 > ids_cap) { status = OR_ERR_CAPACITY; goto out; }
                ids[w++] = kmer_lut[index];
            } else {
                if (w + k > ids_cap) { status = OR_ERR_CAPACITY; goto out; }
                for (int i = 0; i < k; ++i) ids[w++] = base_ids[digit[t + i]];
            }
        }
        for (; t < L; ++t) {  /* the tail */
            if (w + 1 > ids_cap) { status = OR_ERR_CAPACITY; goto out; }
            ids[w++] = base_ids[digit[t]];
        }
    }
    offsets[n_rec] = w;
    *n_ids_out = w;
    *n_rec_out = n_rec;
out:
    free(digit); free(rs); free(hdr);
    return status;
}

/* ---------------------------------------------------- reverse complement */

static uint8_t complement(uint8_t b) {
    static const char from[] = "ACGTRYKMBVDHacgtrykmbvdh";
    static const char to[] = "TGCAYRMKVBHDtgcayrmkvbhd";
    for (int i = 0; from[i]; ++i)
        if ((uint8_t)from[i] == b) return (uint8_t)to[i];
    return b;
}

/* C18: reverse complement of every record [seq_offsets[r], seq_offsets[r+1]). */
int oracle_revcomp(const uint8_t *in, int64_t n, const int64_t *seq_offsets, int64_t n_seq,
                   uint8_t *out) {
    if (n < 0 || n_seq < 0 || !seq_offsets || seq_offsets[0] != 0 || seq_offsets[n_seq] != n)
        return OR_ERR_ARG;
    for (int64_t r = 0; r < n_seq; ++r) {
        const int64_t s = seq_offsets[r], e = seq_offsets[r + 1];
        if (e < s) return OR_ERR_ARG;
        for (int64_t i = s; i < e; ++i) out[s + e - 1 - i] = complement(in[i]);
    }
    return OR_OK;
}

/* -------------------------------------------------------------- decode */

/* Write the bases a BPE token stands for (recursively through the merge
 * table).  Returns the number of bytes written, or -1 if cap is too small. */
static int64_t bpe_token_text(const int32_t *merges, int32_t m, int32_t id, char *out, int64_t cap) {
    if (id >= 0 && id < 4) {
        if (cap < 1) return -1;
        out[0] = "ACGT"[id];
        return 1;
    }
    if (id == 4 + m) {
        if (cap < 1) return -1;
        out[0] = 'N';
        return 1;
    }
    if (id < 4 || id >= 4 + m) return -1;
    int64_t a = bpe_token_text(merges, m, merges[2 * (id - 4)], out, cap);
    if (a < 0) return -1;
    int64_t b = bpe_token_text(merges, m, merges[2 * (id - 4) + 1], out + a, cap - a);
    return b < 0 ? -1 : a + b;
}

/* Decode ids back to text: mode 0 uses the default table's inverse (A C G T
 * N), mode 1 writes k bases per k-mer id and '?' for UNK, mode 2 expands
 * merges, mode 3 (one record of overlapping k-mers) writes the first k-mer's
 * k bases and then the last base of each next one.  Returns the text length
 * or -1. */
int64_t oracle_decode(int mode, int k, const int32_t *merges, int32_t n_merges,
                      const int32_t *ids, int64_t n_ids, char *out, int64_t cap) {
    int64_t w = 0;
    for (int64_t t = 0; t < n_ids; ++t) {
        int32_t id = ids[t];
        if (mode == OR_CHAR) {
            if (w + 1 > cap || id < 0 || id > 4) return -1;
            out[w++] = "ACGTN"[id];
        } else if (mode == OR_KMER_OVL && t > 0) {
            int64_t unk = (int64_t)1 << (2 * k);
            if (w + 1 > cap || id < 0 || id > unk) return -1;
            out[w++] = id == unk ? '?' : "ACGT"[id & 3];
        } else if (mode == OR_KMER || mode == OR_KMER_OVL) {
            int64_t unk = (int64_t)1 << (2 * k);
            if (id == unk) {
                if (w + 1 > cap) return -1;
                out[w++] = '?';
                continue;
            }
            if (id < 0 || id > unk || w + k > cap) return -1;
            for (int i = 0; i < k; ++i) out[w + i] = "ACGT"[(id >> (2 * (k - 1 - i))) & 3];
            w += k;
        } else {
            int64_t m = bpe_token_text(merges, n_merges, id, out + w, cap - w);
            if (m < 0) return -1;
            w += m;
        }
    }
    return w;
}

/* C17: single-nucleotide ids through the inverse of a 256-entry table. */
int64_t oracle_decode_lut(const int32_t *lut, const int32_t *ids, int64_t n_ids, char *out,
                          int64_t cap) {
    int order[256 + 62 + 5], n_order = 0;
    const char *first = "ACGTN";
    for (int i = 0; first[i]; ++i) order[n_order++] = (uint8_t)first[i];
    for (int c = 'A'; c <= 'Z'; ++c) order[n_order++] = c;
    for (int c = 'a'; c <= 'z'; ++c) order[n_order++] = c;
    for (int c = 0; c < 256; ++c) order[n_order++] = c;
    if (n_ids > cap) return -1;
    for (int64_t t = 0; t < n_ids; ++t) {
        int found = -1;
        for (int i = 0; i < n_order && found < 0; ++i)
            if (lut[order[i]] == ids[t]) found = order[i];
        if (found < 0 || ids[t] < 0) return -1;
        out[t] = (char)found;
    }
    return n_ids;
}

/* C17: table-driven k-mer ids back to text. */
int64_t oracle_decode_ktab(int k, const int32_t *kmer_lut, const int32_t *base_ids,
                           const int32_t *ids, int64_t n_ids, char *out, int64_t cap) {
    if (k < 1 || k > 10) return -1;
    int64_t n_index = 1;
    for (int i = 0; i < k; ++i) n_index *= 5;
    int64_t w = 0;
    for (int64_t t = 0; t < n_ids; ++t) {
        const int32_t v = ids[t];
        int64_t index = -1;
        for (int64_t x = 0; x < n_index && index < 0 && v >= 0; ++x)
            if (kmer_lut[x] == v) index = x;
        if (index >= 0) {
            if (w + k > cap) return -1;
            for (int i = k - 1; i >= 0; --i) {
                out[w + i] = "ACGTN"[index % 5];
                index /= 5;
            }
            w += k;
            continue;
        }
        int d = -1;
        for (int x = 0; x < 5 && d < 0; ++x)
            if (base_ids[x] == v && v >= 0) d = x;
        if (d < 0 || w + 1 > cap) return -1;
        out[w++] = "ACGTN"[d];
    }
    return w;
}
