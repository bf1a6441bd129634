// server.cu -- the serving loop: tokenization requests of mixed modes and
// sizes arrive at any time; a worker thread admits them under a device-memory
// budget, packs the admitted requests of one mode into a batch (each request
// is one record of the batch), and launches the batch on one of several
// streams while earlier batches are still running (continuous batching).
// Tables, staging and outputs stay on the device; a request's ids stay in
// the device arena until the caller releases it.  The paper names serving as
// a target use of its layer (Sec. 4.4) without giving a design.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handle.h"

namespace {

double now_us() {
    return std::chrono::duration<double, std::micro>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// First-fit allocator over one address range (offsets; 256-byte granules).
class RangeAlloc {
  public:
    void init(long long size) {
        free_.clear();
        free_[0] = size;
        used_ = 0;
    }
    long long alloc(long long n) {
        n = (n + 255) & ~255ll;
        if (n == 0) n = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const long long off = it->first, rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                used_ += n;
                return off;
            }
        }
        return -1;
    }
    void release(long long off, long long n) {
        n = (n + 255) & ~255ll;
        if (n == 0) n = 256;
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    long long used() const { return used_; }

  private:
    std::map<long long, long long> free_;
    long long used_ = 0;
};

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3 };

struct Request {
    uint64_t id;
    int mode;
    long long n;
    long long host_off;  // in the pinned arena
    double t_submit;
    double t_done = 0;
    int state = RQ_QUEUED;
    int batch = -1;
    long long ids_at = 0;  // device offset (bytes) of its ids in the device arena
    long long n_ids = 0;
    bool released = false;
};

struct Batch {
    bool live = false;
    int mode = 0, slot = 0;
    std::vector<uint64_t> reqs;
    long long in_off = 0, in_bytes = 0;     // device arena: bytes + seq offsets
    long long out_off = 0, out_bytes = 0;   // device arena: ids + id offsets + totals
    long long n_bytes = 0;
    int n_unreleased = 0;
    cudaEvent_t done = nullptr;
    long long *h_offs = nullptr;            // pinned: seq offsets in, id offsets back
    int *h_status = nullptr;                // pinned: the handle's device status, copied back
    bool launch_failed = false;             // dnatok_encode refused the batch on the host
    long long offs_cap = 0;
};

}  // namespace

struct dnatok_server {
    dnatok_server_cfg cfg;
    int n_slots = 4;
    std::vector<dnatok_handle *> handles;  // [slot * 3 + mode]
    std::vector<cudaStream_t> streams;     // per slot
    std::vector<int> slot_busy;
    uint8_t *d_arena = nullptr;
    RangeAlloc dev;
    uint8_t *h_arena = nullptr;
    RangeAlloc host;
    long long host_size = 0;

    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    std::unordered_map<uint64_t, Request> reqs;
    std::deque<uint64_t> queue[3];
    std::vector<Batch> batches;
    uint64_t next_id = 1;
    long long batches_launched = 0;
    std::string error;
    // failure injection for tests (dnatok_server_inject): the next
    // inject_count batches fail as `inject_kind` says
    int inject_kind = 0, inject_count = 0;
};

using namespace dnatok;

namespace {

const int kInjectedDeviceError = DEV_TIMEOUT;

// Worker-side: finish batches whose event fired.  Called with mu held.
void reap(dnatok_server *S) {
    for (size_t b = 0; b < S->batches.size(); ++b) {
        Batch &B = S->batches[b];
        if (!B.live || B.slot < 0) continue;
        const cudaError_t q = cudaEventQuery(B.done);
        if (q == cudaErrorNotReady) continue;
        const double t = now_us();
        const bool dev_error = (q == cudaSuccess && *B.h_status != 0);
        const bool ok = (q == cudaSuccess && !B.launch_failed && !dev_error);
        if (dev_error) {
            // the handle's status word (and, for a look-back that stopped
            // early, its tile counters) must be clear before its next batch;
            // the slot's stream orders this before anything launched later
            dnatok_handle *h = S->handles[B.slot * 3 + B.mode];
            cudaStream_t st = S->streams[B.slot];
            cudaMemsetAsync(h->d_status, 0, sizeof(int), st);
            cudaMemsetAsync(h->d_counter, 0, 2 * sizeof(unsigned long long), st);
        }
        for (size_t i = 0; i < B.reqs.size(); ++i) {
            Request &R = S->reqs[B.reqs[i]];
            R.state = ok ? RQ_DONE : RQ_FAILED;
            R.t_done = t;
            R.ids_at = B.out_off + 4 * B.h_offs[i];
            R.n_ids = B.h_offs[i + 1] - B.h_offs[i];
            S->host.release(R.host_off, R.n);
        }
        S->dev.release(B.in_off, B.in_bytes);
        B.in_bytes = 0;
        S->slot_busy[B.slot] = 0;
        B.slot = -1;  // done; the output stays until every request is released
        if (B.n_unreleased == 0) {
            S->dev.release(B.out_off, B.out_bytes);
            B.live = false;
        }
    }
}

// Worker-side: form and launch batches while slots and memory allow.
void admit(dnatok_server *S) {
    for (int round = 0; round < 3; ++round) {
        for (int mode = 0; mode < 3; ++mode) {
            std::deque<uint64_t> &Q = S->queue[mode];
            if (Q.empty()) continue;
            int slot = -1;
            for (int i = 0; i < S->n_slots; ++i)
                if (!S->slot_busy[i]) {
                    slot = i;
                    break;
                }
            if (slot < 0) return;
            // take requests FIFO up to the batch size
            std::vector<uint64_t> take;
            long long nb = 0, ob = 0;
            for (uint64_t id : Q) {
                const Request &R = S->reqs[id];
                if (!take.empty() && (nb + R.n > S->cfg.max_batch_bytes ||
                                      (long long)take.size() >= S->cfg.max_batch_requests))
                    break;
                take.push_back(id);
                nb += R.n;
            }
            const long long nr = (long long)take.size();
            dnatok_handle *h = S->handles[slot * 3 + mode];
            {
                int64_t cap = 0;
                dnatok_max_tokens(h, nb, nr, &cap);  // what dnatok_encode will ask for
                ob = cap;
            }
            const long long in_bytes = ((nb + 15) & ~15ll) + 8 * (nr + 1);
            const long long ids_bytes = (4 * (ob + 4) + 15) & ~15ll;  // keeps the int64s aligned
            const long long out_bytes = ids_bytes + 8 * (nr + 1) + 16 + 64;
            const long long in_off = S->dev.alloc(in_bytes);
            if (in_off < 0) continue;  // over budget: wait for completions
            const long long out_off = S->dev.alloc(out_bytes);
            if (out_off < 0) {
                S->dev.release(in_off, in_bytes);
                continue;
            }
            // a free batch record
            int bi = -1;
            for (size_t i = 0; i < S->batches.size(); ++i)
                if (!S->batches[i].live) {
                    bi = (int)i;
                    break;
                }
            if (bi < 0) {
                S->batches.emplace_back();
                bi = (int)S->batches.size() - 1;
                Batch &NB = S->batches[bi];
                cudaEventCreateWithFlags(&NB.done, cudaEventDisableTiming);
                cudaHostAlloc(&NB.h_status, sizeof(int), cudaHostAllocDefault);
            }
            Batch &B = S->batches[bi];
            if (B.offs_cap < nr + 1) {
                if (B.h_offs) cudaFreeHost(B.h_offs);
                B.offs_cap = nr + 1 + 64;
                cudaHostAlloc(&B.h_offs, 8 * B.offs_cap, cudaHostAllocDefault);
            }
            B.live = true;
            B.mode = mode;
            B.slot = slot;
            B.reqs = take;
            B.in_off = in_off;
            B.in_bytes = in_bytes;
            B.out_off = out_off;
            B.out_bytes = out_bytes;
            B.n_bytes = nb;
            B.n_unreleased = (int)nr;
            for (long long i = 0; i < nr; ++i) Q.pop_front();
            S->slot_busy[slot] = 1;
            cudaStream_t st = S->streams[slot];
            uint8_t *d_in = S->d_arena + in_off;
            long long *d_so = reinterpret_cast<long long *>(d_in + ((nb + 15) & ~15ll));
            int32_t *d_ids = reinterpret_cast<int32_t *>(S->d_arena + out_off);
            long long *d_io = reinterpret_cast<long long *>(S->d_arena + out_off + ids_bytes);
            long long *d_tot = d_io + (nr + 1);
            long long pos = 0;
            B.h_offs[0] = 0;
            for (long long i = 0; i < nr; ++i) {
                Request &R = S->reqs[take[i]];
                R.state = RQ_RUNNING;
                R.batch = bi;
                if (R.n) cudaMemcpyAsync(d_in + pos, S->h_arena + R.host_off, R.n,
                                         cudaMemcpyHostToDevice, st);
                pos += R.n;
                B.h_offs[i + 1] = pos;
            }
            cudaMemcpyAsync(d_so, B.h_offs, 8 * (nr + 1), cudaMemcpyHostToDevice, st);
            int inject = 0;
            if (S->inject_count > 0) {
                inject = S->inject_kind;
                --S->inject_count;
            }
            if (inject == 2)  // a device-side error, as a bounded wait that ran out records it
                cudaMemcpyAsync(h->d_status, &kInjectedDeviceError, sizeof(int),
                                cudaMemcpyHostToDevice, st);
            dnatok_status rc =
                inject == 1 ? DNATOK_ERR_STATE
                            : dnatok_encode(h, d_in, nb, reinterpret_cast<int64_t *>(d_so), nr,
                                            d_ids, ob + 4, reinterpret_cast<int64_t *>(d_io),
                                            nr + 1, reinterpret_cast<int64_t *>(d_tot),
                                            reinterpret_cast<dnatok_cuda_stream>(st));
            // the id offsets come back to the same pinned array (after the
            // kernel has read the sequence offsets it was given)
            cudaMemcpyAsync(B.h_offs, d_io, 8 * (nr + 1), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(B.h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
            cudaEventRecord(B.done, st);
            // a refusal on the host is kept apart from the status word that
            // the copy above writes back
            B.launch_failed = (rc != DNATOK_OK);
            if (rc != DNATOK_OK) S->error = inject == 1 ? "injected launch failure" : h->last_error;
            ++S->batches_launched;
        }
    }
}

void worker_main(dnatok_server *S) {
    cudaSetDevice(S->handles[0]->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        reap(S);
        admit(S);
        bool inflight = false;
        for (auto &B : S->batches)
            if (B.live && B.slot >= 0) inflight = true;
        bool queued = !S->queue[0].empty() || !S->queue[1].empty() || !S->queue[2].empty();
        if (inflight) {
            S->cv.wait_for(lk, std::chrono::microseconds(20));
        } else if (!queued) {
            S->cv.wait(lk);
        } else {
            // queued but nothing running: memory is held by unreleased outputs
            S->cv.wait_for(lk, std::chrono::microseconds(200));
        }
    }
}

void server_free(dnatok_server *S) {
    for (auto &B : S->batches) {
        if (B.done) cudaEventDestroy(B.done);
        if (B.h_offs) cudaFreeHost(B.h_offs);
        if (B.h_status) cudaFreeHost(B.h_status);
    }
    for (auto h : S->handles) dnatok_destroy(h);
    for (auto s : S->streams) cudaStreamDestroy(s);
    cudaFree(S->d_arena);
    if (S->h_arena) cudaFreeHost(S->h_arena);
    delete S;
}

}  // namespace

extern "C" {

dnatok_status dnatok_server_create(const dnatok_server_cfg *cfg, dnatok_server **out) {
    if (!cfg || !out) return DNATOK_ERR_ARG;
    *out = nullptr;
    if (cfg->budget_bytes < (1 << 20) || cfg->host_arena_bytes < (1 << 20) ||
        cfg->max_batch_bytes < 1 || cfg->max_batch_requests < 1 || cfg->n_slots < 1 ||
        cfg->n_slots > 16 || cfg->kmer_k < 1 || cfg->kmer_k > DNATOK_MAX_K)
        return DNATOK_ERR_ARG;
    dnatok_server *S = new (std::nothrow) dnatok_server();
    if (!S) return DNATOK_ERR_NOMEM;
    S->cfg = *cfg;
    S->n_slots = cfg->n_slots;
    // one request of max_batch_bytes must fit the budget on its own, or it
    // could never be admitted
    dnatok_tables none{nullptr, nullptr, 0, nullptr, nullptr};
    dnatok_tables bpe{nullptr, cfg->merges, cfg->n_merges, nullptr, nullptr};
    for (int slot = 0; slot < S->n_slots; ++slot) {
        for (int mode = 0; mode < 3; ++mode) {
            dnatok_handle *h = nullptr;
            dnatok_status st;
            if (mode == DNATOK_BPE && !cfg->merges && cfg->n_merges > 0) st = DNATOK_ERR_TABLE;
            else
                st = dnatok_create(&h, (dnatok_mode)mode, mode == DNATOK_KMER ? cfg->kmer_k : 1,
                                   mode == DNATOK_BPE ? &bpe : &none, DNATOK_RAW);
            if (st == DNATOK_OK)
                st = dnatok_reserve(h, cfg->max_batch_bytes + (1 << 20), cfg->max_batch_requests);
            if (st != DNATOK_OK) {
                if (h) dnatok_destroy(h);
                server_free(S);
                return st;
            }
            S->handles.push_back(h);
        }
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            server_free(S);
            return DNATOK_ERR_CUDA;
        }
        S->streams.push_back(s);
        S->slot_busy.push_back(0);
    }
    {
        long long worst = 0;
        for (int mode = 0; mode < 3; ++mode) {
            int64_t cap = 0;
            dnatok_max_tokens(S->handles[mode], cfg->max_batch_bytes, 1, &cap);
            const long long in_b = ((cfg->max_batch_bytes + 15) & ~15ll) + 16;
            const long long out_b = ((4 * (cap + 4) + 15) & ~15ll) + 16 + 16 + 64;
            const long long f = ((in_b + 255) & ~255ll) + ((out_b + 255) & ~255ll);
            if (f > worst) worst = f;
        }
        if (worst > cfg->budget_bytes) {
            server_free(S);
            return DNATOK_ERR_BUDGET;
        }
    }
    if (cudaMalloc(&S->d_arena, (size_t)cfg->budget_bytes) != cudaSuccess ||
        cudaHostAlloc(&S->h_arena, (size_t)cfg->host_arena_bytes, cudaHostAllocDefault) !=
            cudaSuccess) {
        server_free(S);
        return DNATOK_ERR_NOMEM;
    }
    S->dev.init(cfg->budget_bytes);
    S->host.init(cfg->host_arena_bytes);
    S->host_size = cfg->host_arena_bytes;
    S->worker = std::thread(worker_main, S);
    *out = S;
    return DNATOK_OK;
}

dnatok_status dnatok_server_submit(dnatok_server *S, int32_t mode, const uint8_t *host_bytes,
                                   int64_t n, uint64_t *req_id) {
    if (!S || !req_id || n < 0 || (n > 0 && !host_bytes) || mode < 0 || mode > 2)
        return DNATOK_ERR_ARG;
    if (mode == DNATOK_BPE && S->cfg.n_merges < 0) return DNATOK_ERR_ARG;
    const double t = now_us();
    std::unique_lock<std::mutex> lk(S->mu);
    if (n > S->cfg.max_batch_bytes) return DNATOK_ERR_CAPACITY;
    const long long off = S->host.alloc(n);
    if (off < 0) return DNATOK_ERR_BUDGET;  // the pinned arena is full: retry later
    if (n) std::memcpy(S->h_arena + off, host_bytes, (size_t)n);
    Request R;
    R.id = S->next_id++;
    R.mode = mode;
    R.n = n;
    R.host_off = off;
    R.t_submit = t;
    S->reqs.emplace(R.id, R);
    S->queue[mode].push_back(R.id);
    *req_id = R.id;
    lk.unlock();
    S->cv.notify_one();
    return DNATOK_OK;
}

dnatok_status dnatok_server_poll(dnatok_server *S, uint64_t req_id, dnatok_server_result *out) {
    if (!S) return DNATOK_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return DNATOK_ERR_UNKNOWN_REQ;
    const Request &R = it->second;
    if (R.state == RQ_QUEUED || R.state == RQ_RUNNING) return DNATOK_PENDING;
    if (R.state == RQ_FAILED) return DNATOK_ERR_CUDA;
    if (out) {
        out->ids_d = reinterpret_cast<const int32_t *>(S->d_arena + R.ids_at);
        out->n_ids = R.n_ids;
        out->latency_us = R.t_done - R.t_submit;
    }
    return DNATOK_OK;
}

dnatok_status dnatok_server_read(dnatok_server *S, uint64_t req_id, int32_t *host_ids,
                                 int64_t capacity, int64_t *n_ids) {
    if (!S || (capacity > 0 && !host_ids)) return DNATOK_ERR_ARG;
    const int32_t *src = nullptr;
    long long n = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(req_id);
        if (it == S->reqs.end()) return DNATOK_ERR_UNKNOWN_REQ;
        const Request &R = it->second;
        if (R.state == RQ_QUEUED || R.state == RQ_RUNNING) return DNATOK_PENDING;
        if (R.state == RQ_FAILED) return DNATOK_ERR_CUDA;
        src = reinterpret_cast<const int32_t *>(S->d_arena + R.ids_at);
        n = R.n_ids;
    }
    if (n_ids) *n_ids = n;
    if (n > capacity) return DNATOK_ERR_CAPACITY;
    if (n && cudaMemcpy(host_ids, src, 4 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return DNATOK_ERR_CUDA;
    return DNATOK_OK;
}

dnatok_status dnatok_server_release(dnatok_server *S, uint64_t req_id) {
    if (!S) return DNATOK_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(req_id);
        if (it == S->reqs.end()) return DNATOK_ERR_UNKNOWN_REQ;
        Request &R = it->second;
        if (R.state != RQ_DONE && R.state != RQ_FAILED) return DNATOK_PENDING;
        Batch &B = S->batches[R.batch];
        if (--B.n_unreleased == 0 && B.slot < 0) {
            S->dev.release(B.out_off, B.out_bytes);
            B.live = false;
        }
        S->reqs.erase(it);
    }
    S->cv.notify_one();
    return DNATOK_OK;
}

dnatok_status dnatok_server_inject(dnatok_server *S, int32_t kind, int32_t count) {
    if (!S || kind < 0 || kind > 2 || count < 0) return DNATOK_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->inject_kind = kind;
    S->inject_count = kind == 0 ? 0 : count;
    return DNATOK_OK;
}

dnatok_status dnatok_server_stats(dnatok_server *S, dnatok_server_counters *out) {
    if (!S || !out) return DNATOK_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out->device_bytes_in_use = S->dev.used();
    out->batches_launched = S->batches_launched;
    long long q = 0, r = 0;
    for (int m = 0; m < 3; ++m) q += (long long)S->queue[m].size();
    for (auto &B : S->batches)
        if (B.live && B.slot >= 0) ++r;
    out->queued = q;
    out->batches_running = r;
    return DNATOK_OK;
}

void dnatok_server_destroy(dnatok_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaDeviceSynchronize();
    server_free(S);
}

}  // extern "C"
