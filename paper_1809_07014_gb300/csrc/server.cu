// Serving loop: k-mer analysis requests arrive at any time, are admitted
// while their estimated device footprint fits the memory budget, and run
// concurrently, each on its own worker thread and CUDA stream, so that the
// device interleaves the kernels of every admitted request (continuous
// batching: a request that arrives while others run starts as soon as a
// worker and memory are free, without waiting for a batch boundary).
//
// Readsets stay resident (the client owns them and may submit the same reads
// at several k, as Algorithm 1 does).  A finished request keeps its analysis
// buffers -- its results -- until the client releases it; released analyses
// go to a pool and serve later requests with the same parameters without new
// allocations, and idle pooled analyses are freed when admission needs room.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "host.h"

using namespace kmer;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    const kmer_readset* rs = nullptr;
    kmer_analysis_params p{};
    uint64_t footprint = 0;
    double t_submit = 0, t_admit = 0, t_start = 0, t_done = 0;
    int status = KMER_OK;
    std::string error;
    kmer_result_view view{};
    kmer_analysis_t* h = nullptr;
    unsigned worker = 0;
    bool admitted = false, done = false;
};

struct Pooled {
    kmer_analysis_t* h;
    kmer_analysis_params p;
    uint64_t bytes;
    unsigned worker;  // an analysis stays on the stream of the worker that created it
};

// Parameters that decide a result (and the partition geometry overrides):
// a pooled analysis with the same ones serves the request after its sizing
// hints (memory budget, distinct keys) are set to the request's.
bool compatible(const kmer_analysis_params& a, const kmer_analysis_params& b) {
    return a.k == b.k && a.min_count == b.min_count && a.qual_offset == b.qual_offset &&
           a.qual_threshold == b.qual_threshold && a.ext_mode == b.ext_mode && a.t_base == b.t_base &&
           a.err_num == b.err_num && a.err_den == b.err_den && a.t_ext == b.t_ext && a.variant == b.variant &&
           a.leaf_bits == b.leaf_bits && a.l1_bits == b.l1_bits && a.flags == b.flags;
}

}  // namespace

struct kmer_server {
    int device = 0;
    uint64_t budget = 0, in_use = 0;
    Clock::time_point t0 = Clock::now();
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;   // waiting for memory, in arrival order
    std::deque<Request*> ready;     // admitted, waiting for a worker
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<Pooled> pool;       // released analyses kept for reuse
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    double ratio[KMER_MAX_K + 1] = {};  // distinct / windows of the last finished request at each k
    uint64_t next_id = 1;
    bool stop = false;
    unsigned running = 0;
    kmer_server_stats st{};

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

// Device bytes an analysis of this readset and k is expected to hold.
uint64_t estimate_footprint(const kmer_readset* rs, const kmer_analysis_params& p, uint64_t budget) {
    const unsigned W = (2 * p.k + 63) / 64;
    const double windows = (double)rs->windows_for(p.k);
    const double records = windows * 8.0 * W * 3.4;          // level-1 + level-2 records with slack
    const double outputs = windows / 4.0 * (8.0 * W + 38.0);  // survivors, first-query estimate
    uint64_t f = (uint64_t)(records + outputs) + (64ull << 20);
    return std::min<uint64_t>(f, budget);
}

// Called with the lock held: admit waiting requests in arrival order while
// they fit.  Idle pooled analyses are evicted to make room; the caller frees
// them after dropping the lock (freeing waits for their stream).
void admit(kmer_server* s, std::vector<kmer_analysis_t*>& evicted) {
    while (!s->pending.empty()) {
        Request* r = s->pending.front();
        while (s->in_use + r->footprint > s->budget && !s->pool.empty()) {
            Pooled victim = s->pool.front();
            s->pool.erase(s->pool.begin());
            s->in_use -= victim.bytes;
            evicted.push_back(victim.h);
        }
        if (s->in_use + r->footprint > s->budget) break;  // wait for a release
        s->pending.pop_front();
        s->in_use += r->footprint;
        r->admitted = true;
        r->t_admit = s->now_ms();
        s->ready.push_back(r);
        s->cv_work.notify_one();
    }
}

void worker(kmer_server* s, unsigned wi) {
    cudaSetDevice(s->device);
    cudaStream_t stream = s->streams[wi];
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_work.wait(lk, [&] { return s->stop || !s->ready.empty(); });
        if (s->stop && s->ready.empty()) return;
        Request* r = s->ready.front();
        s->ready.pop_front();
        // an idle analysis with the same parameters carries its buffers over
        kmer_analysis_t* h = nullptr;
        for (size_t i = 0; i < s->pool.size(); ++i) {
            if (s->pool[i].worker == wi && compatible(s->pool[i].p, r->p)) {
                h = s->pool[i].h;
                s->in_use -= s->pool[i].bytes;  // the request's footprint now covers it
                s->pool.erase(s->pool.begin() + (long)i);
                break;
            }
        }
        r->t_start = s->now_ms();
        s->running++;
        s->st.peak_running = std::max(s->st.peak_running, s->running);
        lk.unlock();
        int rc = KMER_OK;
        if (!h) {
            rc = kmer_analysis_create(&r->p, stream, &h);
        } else {
            analysis_set_sizing(h, r->p.memory_budget, r->p.distinct_hint);
            rc = kmer_analysis_reset(h);
        }
        if (rc == KMER_OK) rc = kmer_analysis_submit(h, r->rs);
        if (rc == KMER_OK) rc = kmer_analysis_query(h, &r->view);
        std::string err = rc == KMER_OK ? std::string() : std::string(kmer_last_error_message());
        lk.lock();
        if (rc == KMER_OK && r->view.windows)
            s->ratio[r->p.k] = (double)r->view.distinct / (double)r->view.windows;
        s->running--;
        r->h = h;
        r->worker = wi;
        r->status = rc;
        r->error = err;
        r->t_done = s->now_ms();
        r->done = true;
        s->st.completed++;
        if (rc != KMER_OK) s->st.failed++;
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

int kmer_server_create(uint64_t memory_budget, uint32_t workers, kmer_server_t** out) {
    if (!out) return fail(KMER_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (workers == 0 || workers > 64) return fail(KMER_ERR_INVALID_ARG, "workers must be in 1..64");
    auto* s = new (std::nothrow) kmer_server;
    if (!s) return fail(KMER_ERR_OOM, "host allocation failed");
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(KMER_ERR_NO_DEVICE, "no CUDA device");
    }
    prepare_pool(s->device);
    if (!memory_budget) memory_budget = (uint64_t)(0.7 * (double)free_device_bytes());
    s->budget = memory_budget;
    s->streams.resize(workers);
    for (unsigned i = 0; i < workers; ++i) {
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (unsigned j = 0; j < i; ++j) cudaStreamDestroy(s->streams[j]);
            delete s;
            return fail(KMER_ERR_CUDA, "cannot create a stream");
        }
    }
    for (unsigned i = 0; i < workers; ++i) s->workers.emplace_back(worker, s, i);
    s->st.workers = workers;
    *out = s;
    return KMER_OK;
}

int kmer_server_submit(kmer_server_t* s, const kmer_readset_t* rs, const kmer_analysis_params* p, uint64_t* id) {
    if (!s || !rs || !p || !id) return fail(KMER_ERR_INVALID_ARG, "NULL argument");
    if (p->k == 0 || p->k > KMER_MAX_K || p->k % 2 == 0 || p->min_count == 0)
        return fail(KMER_ERR_INVALID_ARG, "invalid parameters");
    if (rs->qual_offset != p->qual_offset || rs->qual_threshold != p->qual_threshold)
        return fail(KMER_ERR_INVALID_ARG, "readset packed with other quality parameters");
    auto r = std::make_unique<Request>();
    std::vector<kmer_analysis_t*> evicted;
    r->rs = rs;
    r->p = *p;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->footprint = estimate_footprint(rs, *p, s->budget);
        if (!r->p.memory_budget || r->p.memory_budget > r->footprint) r->p.memory_budget = r->footprint;
        // distinct keys expected from the last request at this k (sizes the partitions)
        if (!r->p.distinct_hint && s->ratio[p->k] > 0.0)
            r->p.distinct_hint = (uint64_t)(1.1 * s->ratio[p->k] * (double)rs->windows_for(p->k)) + 1;
        r->id = s->next_id++;
        r->t_submit = s->now_ms();
        *id = r->id;
        s->pending.push_back(r.get());
        s->reqs.emplace(r->id, std::move(r));
        s->st.submitted++;
        admit(s, evicted);
    }
    for (auto* h : evicted) kmer_analysis_destroy(h);
    return KMER_OK;
}

int kmer_server_poll(kmer_server_t* s, uint64_t id, int* done) {
    if (!s || !done) return fail(KMER_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(KMER_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)id);
    *done = it->second->done ? 1 : 0;
    return KMER_OK;
}

int kmer_server_wait(kmer_server_t* s, uint64_t id, kmer_result_view* out, kmer_request_info* info) {
    if (!s) return fail(KMER_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(KMER_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)id);
    Request* r = it->second.get();
    s->cv_done.wait(lk, [&] { return r->done; });
    if (out) *out = r->view;
    if (info) {
        info->id = r->id;
        info->status = r->status;
        info->t_submit_ms = r->t_submit;
        info->t_admit_ms = r->t_admit;
        info->t_start_ms = r->t_start;
        info->t_done_ms = r->t_done;
        info->footprint_bytes = r->footprint;
    }
    if (r->status != KMER_OK) return fail(r->status, "request %llu: %s", (unsigned long long)id, r->error.c_str());
    return KMER_OK;
}

int kmer_server_copy_results(kmer_server_t* s, uint64_t id, uint64_t* keys, uint32_t* count, uint32_t* ext,
                             uint8_t* cls, uint64_t capacity) {
    if (!s) return fail(KMER_ERR_INVALID_ARG, "NULL server");
    kmer_analysis_t* h = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return fail(KMER_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)id);
        if (!it->second->done || it->second->status != KMER_OK)
            return fail(KMER_ERR_BAD_STATE, "request %llu has no results", (unsigned long long)id);
        h = it->second->h;
    }
    return kmer_analysis_copy_results(h, keys, count, ext, cls, capacity);
}

int kmer_server_release(kmer_server_t* s, uint64_t id) {
    if (!s) return fail(KMER_ERR_INVALID_ARG, "NULL server");
    std::vector<kmer_analysis_t*> evicted;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(KMER_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)id);
    Request* r = it->second.get();
    if (!r->done) return fail(KMER_ERR_BAD_STATE, "request %llu is still running", (unsigned long long)id);
    s->in_use -= r->footprint;
    if (r->h) {
        kmer_analysis_stats st;
        kmer_analysis_get_stats(r->h, &st);
        kmer_analysis_reset(r->h);
        // keep the analysis (and its buffers) for a later request with the same parameters
        s->pool.push_back({r->h, r->p, st.device_bytes, r->worker});
        s->in_use += st.device_bytes;
    }
    s->reqs.erase(it);
    admit(s, evicted);
    lk.unlock();
    for (auto* h : evicted) kmer_analysis_destroy(h);
    return KMER_OK;
}

int kmer_server_get_stats(kmer_server_t* s, kmer_server_stats* out) {
    if (!s || !out) return fail(KMER_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->bytes_in_use = s->in_use;
    out->budget = s->budget;
    out->pending = (uint32_t)s->pending.size();
    out->running = s->running;
    out->pooled = (uint32_t)s->pool.size();
    return KMER_OK;
}

int kmer_server_destroy(kmer_server_t* s) {
    if (!s) return KMER_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // finish what was admitted; drop what never was
        s->cv_done.wait(lk, [&] { return s->ready.empty() && s->running == 0; });
        s->stop = true;
        s->cv_work.notify_all();
    }
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->reqs)
        if (kv.second->h) kmer_analysis_destroy(kv.second->h);
    for (auto& pl : s->pool) kmer_analysis_destroy(pl.h);
    for (auto st : s->streams) cudaStreamDestroy(st);
    delete s;
    return KMER_OK;
}

}  // extern "C"
