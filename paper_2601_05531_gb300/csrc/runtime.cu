// runtime.cu -- CUDA-graph capture of encodes and the launch-shape autotuner.
//
// Graphs: any sequence of dnatok_encode calls (and other stream work) issued
// between dnatok_graph_begin and dnatok_graph_end on one stream becomes one
// graph that replays with a single launch.  Encodes notice the capture and
// clear the look-back descriptors they use inside the graph, so every replay
// starts clean.  Workspace must be reserved first (dnatok_reserve): nothing
// may allocate under capture.
//
// Autotuner: times every supported launch shape of the tokenization kernel
// (tile bytes, threads, tiles per chunk, resident CTAs per SM) -- for BPE
// handles the segment size of the merge pass, and for k-mer handles whose RAW
// encodes take the direct kernel its slots per step, ring depth and resident
// CTAs per SM -- on the caller's own input,
// keeps the fastest on the handle, and remembers it in an optional text
// cache keyed by GPU name, mode, k, format and input size class.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "handle.h"

struct dnatok_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace dnatok;

namespace {

struct Candidate {
    int a, b, c, d;  // tile, threads, ctas_per_sm, chunk_tiles  |  BPE: seg, halo(-1 = default)
};

// Does a RAW encode on this handle take the direct k-mer kernel?
bool tunes_direct(const dnatok_handle *h, long long n_seq) {
    return h->mode == DNATOK_KMER && h->k >= 2 && h->fmt == DNATOK_RAW && h->direct &&
           direct_eligible(MODE_KMER, n_seq, h->lut_host);
}

std::string cache_key(const dnatok_handle *h, long long n_bytes, bool direct) {
    cudaDeviceProp prop;
    std::string gpu = "gpu";
    if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) gpu = prop.name;
    for (auto &ch : gpu)
        if (ch == ' ') ch = '_';
    int cls = 0;
    while ((1ll << (cls + 1)) <= n_bytes) ++cls;
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s mode=%d k=%d fmt=%d size=2^%d%s", gpu.c_str(), h->mode,
                  h->k, h->fmt, cls, direct ? " direct" : "");
    return buf;
}

bool cache_lookup(const char *path, const std::string &key, Candidate *c) {
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool hit = false;
    while (std::fgets(line, sizeof(line), f)) {
        const char *sep = std::strstr(line, " -> ");
        if (!sep || std::string(line, sep - line) != key) continue;
        Candidate t;
        if (std::sscanf(sep + 4, "%d %d %d %d", &t.a, &t.b, &t.c, &t.d) == 4) {
            *c = t;  // the last entry for a key wins
            hit = true;
        }
    }
    std::fclose(f);
    return hit;
}

void cache_store(const char *path, const std::string &key, const Candidate &c, float ms) {
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s -> %d %d %d %d   # %.4f ms\n", key.c_str(), c.a, c.b, c.c, c.d, ms);
    std::fclose(f);
}

dnatok_status apply(dnatok_handle *h, const Candidate &c, bool direct) {
    if (direct) return dnatok_set_direct_launch(h, c.a, c.b, c.c);  // slots, ring, CTAs per SM
    if (h->mode == DNATOK_BPE) {
        int seg = 0, halo = 0;
        bpe_get_launch(h, &seg, &halo);
        return bpe_set_launch(h, c.a, c.b >= 0 ? c.b : halo);
    }
    dnatok_launch_cfg cfg{c.a, c.b, c.c, c.d};
    return dnatok_set_launch(h, &cfg);
}

}  // namespace

extern "C" {

dnatok_status dnatok_graph_begin(dnatok_handle *h, dnatok_cuda_stream stream) {
    if (!h) return DNATOK_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!s) return fail(h, DNATOK_ERR_ARG, "capture needs a non-default stream");
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaStreamBeginCapture");
    return DNATOK_OK;
}

dnatok_status dnatok_graph_end(dnatok_handle *h, dnatok_cuda_stream stream, dnatok_graph **out) {
    if (!h || !out) return DNATOK_ERR_ARG;
    *out = nullptr;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) return fail_cuda(h, e, "cudaStreamEndCapture");
    dnatok_graph *G = new (std::nothrow) dnatok_graph();
    if (!G) {
        cudaGraphDestroy(g);
        return fail(h, DNATOK_ERR_NOMEM, "host allocation failed");
    }
    G->graph = g;
    e = cudaGraphInstantiate(&G->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        delete G;
        return fail_cuda(h, e, "cudaGraphInstantiate");
    }
    *out = G;
    return DNATOK_OK;
}

dnatok_status dnatok_graph_launch(dnatok_graph *g, dnatok_cuda_stream stream) {
    if (!g) return DNATOK_ERR_ARG;
    return cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
               ? DNATOK_OK
               : DNATOK_ERR_CUDA;
}

void dnatok_graph_destroy(dnatok_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

dnatok_status dnatok_autotune(dnatok_handle *h, const uint8_t *bytes_d, int64_t n_bytes,
                              const int64_t *seq_offsets_d, int64_t n_seq, int32_t *ids_out_d,
                              int64_t ids_capacity, int64_t *id_offsets_d,
                              int64_t offsets_capacity, int32_t reps, const char *cache_path,
                              dnatok_launch_cfg *best_out, float *best_ms_out) {
    if (!h || reps < 1) return DNATOK_ERR_ARG;
    const bool direct = tunes_direct(h, n_seq);
    const std::string key = cache_key(h, n_bytes, direct);
    Candidate best{};
    float best_ms = -1.f;
    if (cache_lookup(cache_path, key, &best)) {
        dnatok_status st = apply(h, best, direct);
        if (st != DNATOK_OK) return st;
    } else {
        std::vector<Candidate> cands;
        if (direct) {
            // slots per step, ring steps, resident CTAs per SM
            const int pairs[3][2] = {{2, 4}, {1, 8}, {4, 2}};
            for (auto &pr : pairs)
                for (int c = 1; c <= 4; ++c) cands.push_back({pr[0], pr[1], c, 0});
        } else if (h->mode == DNATOK_BPE) {
            for (int seg : {256, 512, 1024, 2048, 4096}) cands.push_back({seg, -1, 0, 0});
        } else {
            const int shapes[4][3] = {{8192, 256, 8}, {16384, 256, 4}, {16384, 256, 8}, {32768, 512, 4}};
            for (auto &sh : shapes)
                for (int c = 1; c <= (sh[0] == 8192 ? 8 : sh[0] == 16384 ? 4 : 2); ++c)
                    cands.push_back({sh[0], sh[1], c, sh[2]});
        }
        cudaStream_t s = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        void *flush = nullptr;
        const size_t flush_bytes = 192ull << 20;  // larger than L2: each rep starts cold
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        if (e == cudaSuccess) e = cudaMalloc(&flush, flush_bytes);
        dnatok_status st = DNATOK_OK;
        if (e != cudaSuccess) st = fail_cuda(h, e, "autotune set-up");
        for (size_t i = 0; st == DNATOK_OK && i < cands.size(); ++i) {
            st = apply(h, cands[i], direct);
            if (st != DNATOK_OK) break;
            float tot = 0.f;
            for (int r = 0; r <= reps && st == DNATOK_OK; ++r) {
                cudaMemsetAsync(flush, r & 0xFF, flush_bytes, s);
                cudaEventRecord(a, s);
                st = dnatok_encode(h, bytes_d, n_bytes, seq_offsets_d, n_seq, ids_out_d,
                                   ids_capacity, id_offsets_d, offsets_capacity, nullptr,
                                   reinterpret_cast<dnatok_cuda_stream>(s));
                cudaEventRecord(b, s);
                if (st == DNATOK_OK) st = dnatok_sync(h, reinterpret_cast<dnatok_cuda_stream>(s));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (r > 0) tot += ms;  // the first run warms up
            }
            if (st != DNATOK_OK) break;
            const float ms = tot / reps;
            if (best_ms < 0.f || ms < best_ms) {
                best_ms = ms;
                best = cands[i];
            }
        }
        if (flush) cudaFree(flush);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (s) cudaStreamDestroy(s);
        if (st != DNATOK_OK) return st;
        st = apply(h, best, direct);
        if (st != DNATOK_OK) return st;
        cache_store(cache_path, key, best, best_ms);
    }
    if (best_out) {
        if (direct) {
            *best_out = dnatok_launch_cfg{512 * h->dshape.slots, 256, h->dshape.ctas_per_sm,
                                          h->dshape.ring};
        } else if (h->mode == DNATOK_BPE) {
            int seg = 0, halo = 0;
            bpe_get_launch(h, &seg, &halo);
            *best_out = dnatok_launch_cfg{seg, halo, 0, 0};
        } else {
            dnatok_get_launch(h, best_out);
        }
    }
    if (best_ms_out) *best_ms_out = best_ms;
    return DNATOK_OK;
}

}  // extern "C"
