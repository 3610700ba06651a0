// Batched k-mer analysis: many independent analyses (different samples, k
// and sizes) run through the same stage kernels in one CUDA graph per wave.
//
// Every stage is one launch over all jobs of a key width (the kernels take a
// device array of job descriptors and map each CTA's work unit to its job),
// so small jobs share the GPU instead of each paying its own launches and
// host round trips.  Jobs are grouped into waves whose scratch fits the
// memory budget; a wave is captured once as a graph (zero the counters,
// scatter, plan level 2, repartition, count/classify/compact) and replayed
// by every run.  Buffers are sized ahead from each job's exact window count
// and its expected distinct / surviving k-mers.  After a wave, while its
// scratch still holds the records, a job whose output or level-2 layout was
// too small is repaired in place: its output (or fallback list) is grown, or
// its leaves get an exact layout from the counts the repartition took, and
// the later stages are re-run for that job alone; the repaired descriptor is
// kept for later runs.  Leaves that did not fit an on-chip table are
// recounted in an HBM table.  Only a job whose level-1 buckets overflowed,
// or that is too large for any wave, runs alone through the regular
// analysis.
#include <chrono>
#include <memory>

#include "host.h"

using namespace kmer;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct BJob {
    const kmer_readset* rs = nullptr;
    kmer_analysis_params p{};
    uint64_t survivors_hint = 0;
    Geometry g{};
    unsigned W = 1, cap_max = 0;
    unsigned long long windows = 0, l1_total = 0, l2_capacity = 0, out_cap = 0;
    unsigned long long basis = 1;  // distinct keys the geometry was planned for
    std::vector<unsigned long long> caps, starts;
    size_t scratch_bytes = 0;
    int wave = -1;            // -1: runs alone through the regular path
    unsigned slot = 0;        // index in its wave's job array
    DevBuf out_keys, out_count, out_ext, out_cls;
    DevBuf fb;                // fallback key ranges
    unsigned fb_cap = 64;
    DevBuf split;             // leaves counted again in key ranges (one entry per leaf at most)
    DevBuf l2_exact;          // exact level-2 layout, once a leaf overflowed its uniform capacity
    unsigned exact_p1 = 0, exact_p2 = 0;  // the geometry that layout belongs to
    DevBuf consts;            // level-1 bucket starts and capacities (fixed for the batch's life)
    Job job{};                // device descriptor (pointers filled per wave)
    kmer_analysis_t* alone = nullptr;  // regular analysis used for this job, if any
    kmer_result_view alone_view{};
    bool used_alone = false;
    unsigned long long n_out = 0, res_windows = 0, res_distinct = 0;
};

struct Wave {
    std::vector<unsigned> ids;  // job indices, grouped by key width
    struct Cls {
        unsigned W, first, count, max_p1, max_p2, cap_max, min_k;
        unsigned long long tiles, leaves;
    };
    std::vector<Cls> classes;
    DevBuf maps;                // per class: tile_off, leaf_off, job_tile_off
    std::vector<size_t> tile_off_at, leaf_off_at, job_tile_off_at;
    DevBuf d_jobs;
    size_t zero_bytes = 0;      // counters zeroed at the start of every run
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct kmer_batch {
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;   // the legacy default stream cannot be captured: a private stream replaces it
    size_t leaf_budget = 0;
    std::vector<BJob> jobs;
    std::vector<Wave> waves;
    DevBuf scratch;             // shared by the waves (they run one after the other)
    DevBuf zero;                // per wave: level-1/2 fill counters (largest wave)
    DevBuf misc;                // one Misc per job
    DevBuf hbm;                 // HBM table for leaves recounted after a wave
    DevBuf one_maps;            // work maps of a single-job re-run: leaf_off[2], job_tile_off[2]
    std::vector<Misc> host_misc;
    kmer_batch_stats st{};
    bool have_result = false;
    size_t budget = 0;
    bool replan = false;        // the last run's counts differ from the plan: re-plan before the next run
};

namespace {

unsigned leaf_cap_for(const kmer_batch* b, unsigned W) { return leaf_table_cap(W, b->leaf_budget); }

int plan_job(kmer_batch* b, BJob& j) {
    const kmer_analysis_params& p = j.p;
    j.W = (2 * p.k + 63) / 64;
    j.windows = j.rs->windows_for(p.k);
    j.cap_max = leaf_cap_for(b, j.W);
    unsigned long long basis = j.windows;
    if (p.distinct_hint) basis = std::min<unsigned long long>(p.distinct_hint, j.windows);
    j.basis = std::max<unsigned long long>(basis, 1);
    // one pass (a batch never splits a job into passes: such jobs run alone)
    j.g = plan_geometry(p.k, std::max<unsigned long long>(j.windows, 1), std::max<unsigned long long>(basis, 1),
                        ~size_t(0) / 4, j.cap_max, p.leaf_bits, p.l1_bits, false);
    const unsigned P1 = 1u << j.g.p1, P = 1u << (j.g.p1 + j.g.p2);
    const unsigned long long mean = (j.windows + P1 - 1) / P1;
    j.caps.assign(P1, mean + mean / 8 + 1024);
    j.starts.assign(P1 + 1, 0);
    for (unsigned i = 0; i < P1; ++i) j.starts[i + 1] = j.starts[i] + j.caps[i];
    j.l1_total = j.starts[P1];
    j.l2_capacity = j.g.p2 ? 2 * (j.l1_total + P) + 257ull * P + 1024 : 0;
    const unsigned long long bound = j.windows / p.min_count + 1024;
    const unsigned long long est = j.survivors_hint ? j.survivors_hint + j.survivors_hint / 4 + 4096
                                                    : j.windows / 4 + 4096;
    j.out_cap = std::min(bound, est);
    size_t s = 0;
    s += align_up(j.l1_total * 8 * j.W + 64);        // level-1 records
    if (j.g.p2) {
        s += align_up(j.l2_capacity * 8 * j.W + 64);  // level-2 records
        s += align_up(P1 * 8) + align_up(P1 * 4) + align_up((P1 + 1) * 8);  // base, leafcap, tile prefix
    }
    j.scratch_bytes = s;
    return KMER_OK;
}

size_t zero_bytes_of(const BJob& j) {
    const unsigned P1 = 1u << j.g.p1, P = 1u << (j.g.p1 + j.g.p2);
    return align_up(P1 * 8) + (j.g.p2 ? align_up((size_t)P * 8) : 0);
}

// Fill the device descriptor of job j for its wave's scratch and counters.
int bind_job(kmer_batch* b, BJob& j, unsigned char* scratch, unsigned char* zero, unsigned idx) {
    const unsigned P1 = 1u << j.g.p1, P = 1u << (j.g.p1 + j.g.p2);
    Job& d = j.job;
    d = Job{};
    d.blocks = j.rs->blocks.as<PackedBlock>();
    d.blk_off = j.rs->blk_off.as<unsigned long long>();
    d.offsets = j.rs->offsets.as<unsigned long long>();
    d.n_reads = j.rs->n_reads;
    d.g = j.g;
    d.pass = 0;
    size_t o = 0;
    d.l1_rec = reinterpret_cast<unsigned long long*>(scratch + o);
    // the repartition's bulk copies start on 16-byte boundaries of this region
    if (reinterpret_cast<uintptr_t>(d.l1_rec) & 15) return fail(KMER_ERR_CUDA, "level-1 records not 16-byte aligned");
    o += align_up(j.l1_total * 8 * j.W + 64);
    // bucket starts and capacities never change: kept in the job's own buffer
    TRY(j.consts.ensure((2 * P1 + 1) * 8));
    unsigned long long* cst = j.consts.as<unsigned long long>();
    CK(cudaMemcpyAsync(cst, j.starts.data(), (P1 + 1) * 8, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(cst + P1 + 1, j.caps.data(), P1 * 8, cudaMemcpyHostToDevice, b->stream));
    d.l1_start = cst;
    d.l1_cap = cst + P1 + 1;
    size_t z = 0;
    d.l1_fill = reinterpret_cast<unsigned long long*>(zero + z);
    z += align_up(P1 * 8);
    if (j.g.p2) {
        d.l2_rec = reinterpret_cast<unsigned long long*>(scratch + o);
        o += align_up(j.l2_capacity * 8 * j.W + 64);
        d.l2_base = reinterpret_cast<unsigned long long*>(scratch + o);
        o += align_up(P1 * 8);
        d.l2_leafcap = reinterpret_cast<unsigned*>(scratch + o);
        o += align_up(P1 * 4);
        d.tile_prefix = reinterpret_cast<unsigned long long*>(scratch + o);
        o += align_up((P1 + 1) * 8);
        d.l2_fill = reinterpret_cast<unsigned long long*>(zero + z);
        z += align_up((size_t)P * 8);
        d.l2_capacity = j.l2_capacity;
        if (j.l2_exact.p && j.exact_p1 == j.g.p1 && j.exact_p2 == j.g.p2) {  // a layout learned by a repair
            d.l2_leaf_start = j.l2_exact.as<unsigned long long>();
            d.l2_capacity = ~0ull;
        }
    }
    d.out_keys = j.out_keys.as<unsigned long long>();
    d.out_count = j.out_count.as<unsigned>();
    d.out_ext = j.out_ext.as<unsigned>();
    d.out_cls = j.out_cls.as<unsigned char>();
    d.out_cap = j.out_cap;
    Misc* m = b->misc.as<Misc>() + idx;
    d.out_n = &m->out_n;
    d.status = &m->status;
    d.stats = m->stats;
    TRY(j.fb.ensure(j.fb_cap * 4ull));
    d.fb_list = j.fb.as<unsigned>();
    d.fb_n = &m->fb_n;
    d.fb_cap = j.fb_cap;
    TRY(j.split.ensure((size_t)P * 4));
    d.split_list = j.split.as<unsigned>();
    d.split_n = &m->split_n;
    d.split_cap = P;
    d.min_count = j.p.min_count;
    d.ext_mode = j.p.ext_mode;
    d.t_base = j.p.t_base;
    d.err_num = j.p.err_num;
    d.err_den = j.p.err_den;
    d.t_ext = j.p.t_ext;
    d.l2_slack_num = 512;
    const double ratio = j.p.distinct_hint && j.windows
                             ? std::min(1.0, 2.5 * (double)j.p.distinct_hint / (double)j.windows + 0.1)
                             : 1.0;
    d.table_ratio_num = (unsigned)(ratio * 65536.0);
    return KMER_OK;
}

int capture_wave(kmer_batch* b, Wave& w) {
    // work maps per key-width class
    std::vector<unsigned long long> host_maps;
    for (auto& c : w.classes) {
        std::vector<unsigned long long> tile_off(1, 0), leaf_off(1, 0);
        for (unsigned i = 0; i < c.count; ++i) {
            const BJob& j = b->jobs[w.ids[c.first + i]];
            tile_off.push_back(tile_off.back() + (j.rs->n_reads + 255) / 256);
            leaf_off.push_back(leaf_off.back() + (1ull << (j.g.p1 + j.g.p2)));
        }
        c.tiles = tile_off.back();
        c.leaves = leaf_off.back();
        w.tile_off_at.push_back(host_maps.size());
        host_maps.insert(host_maps.end(), tile_off.begin(), tile_off.end());
        w.leaf_off_at.push_back(host_maps.size());
        host_maps.insert(host_maps.end(), leaf_off.begin(), leaf_off.end());
        w.job_tile_off_at.push_back(host_maps.size());
        host_maps.insert(host_maps.end(), c.count + 1, 0ull);
    }
    TRY(w.maps.ensure(host_maps.size() * 8));
    CK(cudaMemcpyAsync(w.maps.p, host_maps.data(), host_maps.size() * 8, cudaMemcpyHostToDevice, b->stream));
    std::vector<Job> descs;
    for (unsigned id : w.ids) descs.push_back(b->jobs[id].job);
    TRY(w.d_jobs.ensure(descs.size() * sizeof(Job)));
    CK(cudaMemcpyAsync(w.d_jobs.p, descs.data(), descs.size() * sizeof(Job), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));

    const Job* dj = w.d_jobs.as<Job>();
    unsigned long long* maps = w.maps.as<unsigned long long>();
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    // the wave's fill counters, then each job's counters (its slot of b->misc)
    cudaError_t e = cudaMemsetAsync(b->zero.p, 0, w.zero_bytes, b->stream);
    for (unsigned id : w.ids)
        if (e == cudaSuccess) e = cudaMemsetAsync(b->misc.as<Misc>() + id, 0, sizeof(Misc), b->stream);
    for (size_t ci = 0; ci < w.classes.size() && e == cudaSuccess; ++ci) {
        const auto& c = w.classes[ci];
        e = launch_scatter(c.W, dj + c.first, maps + w.tile_off_at[ci], c.count, c.tiles, c.max_p1, c.min_k, false,
                           b->stream);
    }
    for (size_t ci = 0; ci < w.classes.size() && e == cudaSuccess; ++ci) {
        const auto& c = w.classes[ci];
        if (!c.max_p2) continue;
        e = launch_l2_plan(dj + c.first, c.count, maps + w.job_tile_off_at[ci], b->stream);
        if (e == cudaSuccess)
            e = launch_repart(c.W, dj + c.first, maps + w.job_tile_off_at[ci], c.count, c.max_p2, b->num_sms,
                              b->stream);
    }
    for (size_t ci = 0; ci < w.classes.size() && e == cudaSuccess; ++ci) {
        const auto& c = w.classes[ci];
        e = launch_leaf(c.W, dj + c.first, maps + w.leaf_off_at[ci], c.count, c.leaves, c.cap_max, b->num_sms,
                        b->stream);
        if (e == cudaSuccess) e = launch_leaf_split(c.W, dj + c.first, c.count, c.cap_max, b->num_sms, b->stream);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(KMER_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&w.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KMER_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return KMER_OK;
}

void destroy_batch(kmer_batch* b) {
    for (auto& w : b->waves)
        if (w.exec) cudaGraphExecDestroy(w.exec);
    for (auto& j : b->jobs)
        if (j.alone) kmer_analysis_destroy(j.alone);
    // buffers are freed in the order of the batch's stream: before that stream goes
    b->jobs.clear();
    b->waves.clear();
    DevBuf* bs[] = {&b->scratch, &b->zero, &b->misc, &b->hbm, &b->one_maps};
    for (auto* x : bs) x->release();
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Plans every job (geometry and buffer sizes from its parameters and
// hints), groups the jobs into waves that fit the budget, binds their
// descriptors and captures one graph per wave.  Called at creation and again
// when a run's counts show that the plan was off.
int build_plan(kmer_batch* b) {
    const unsigned n_jobs = (unsigned)b->jobs.size();
    for (auto& w : b->waves)
        if (w.exec) cudaGraphExecDestroy(w.exec);
    b->waves.clear();
    for (auto& j : b->jobs) {
        j.wave = -1;
        j.slot = 0;
        TRY(plan_job(b, j));
    }
    const size_t budget = b->budget;
    // persistent per-job state: outputs, counters, fallback lists.  When the
    // exact upper bound (windows / min_count survivors) of every job fits in
    // 40% of the budget it is used, so no job can overflow its output.
    size_t persistent = 0, exact = 0;
    for (auto& j : b->jobs) exact += (j.windows / j.p.min_count + 1024) * (8ull * j.W + 4 + 32 + 2);
    for (auto& j : b->jobs) {
        if (exact <= budget / 5 * 2) j.out_cap = j.windows / j.p.min_count + 1024;
        persistent += j.out_cap * (8ull * j.W + 4 + 32 + 2);
    }
    if (persistent >= budget) return fail(KMER_ERR_OOM, "batch outputs alone need %zu bytes", persistent);
    const size_t scratch_budget = budget - persistent;
    // waves: jobs in the given order, as many as fit; a job larger than the budget runs alone
    size_t max_scratch = 0, max_zero = 0;
    {
        Wave cur;
        size_t cur_bytes = 0, cur_zero = 0;
        auto close = [&]() {
            if (cur.ids.empty()) return;
            cur.zero_bytes = cur_zero;
            max_scratch = std::max(max_scratch, cur_bytes);
            max_zero = std::max(max_zero, cur_zero);
            b->waves.push_back(std::move(cur));
            cur = Wave();
            cur_bytes = cur_zero = 0;
        };
        for (unsigned i = 0; i < n_jobs; ++i) {
            BJob& j = b->jobs[i];
            if (j.windows == 0) continue;  // nothing to count
            if (j.scratch_bytes > scratch_budget) continue;  // runs alone (passes)
            if (cur_bytes + j.scratch_bytes > scratch_budget) close();
            cur.ids.push_back(i);
            cur_bytes += j.scratch_bytes;
            cur_zero += zero_bytes_of(j);
        }
        close();
    }
    TRY(b->misc.ensure(std::max<size_t>(1, n_jobs) * sizeof(Misc)));
    TRY(b->one_maps.ensure(4 * 8));
    TRY(b->scratch.ensure(std::max<size_t>(max_scratch, 256)));
    TRY(b->zero.ensure(std::max<size_t>(max_zero, 256)));
    b->host_misc.resize(n_jobs);
    for (unsigned wi = 0; wi < b->waves.size(); ++wi) {
        Wave& w = b->waves[wi];
        // group by key width: classes are contiguous ranges of w.ids
        std::stable_sort(w.ids.begin(), w.ids.end(),
                         [&](unsigned x, unsigned y) { return b->jobs[x].W < b->jobs[y].W; });
        size_t so = 0, zo = 0;
        for (unsigned s = 0; s < w.ids.size(); ++s) {
            BJob& j = b->jobs[w.ids[s]];
            j.wave = (int)wi;
            j.slot = s;
            TRY(j.out_keys.ensure(j.out_cap * 8 * j.W + 16));
            TRY(j.out_count.ensure(j.out_cap * 4 + 16));
            TRY(j.out_ext.ensure(j.out_cap * 32 + 16));
            TRY(j.out_cls.ensure(j.out_cap * 2 + 16));
            TRY(bind_job(b, j, b->scratch.as<unsigned char>() + so, b->zero.as<unsigned char>() + zo, w.ids[s]));
            so += j.scratch_bytes;
            zo += zero_bytes_of(j);
            if (w.classes.empty() || w.classes.back().W != j.W)
                w.classes.push_back({j.W, s, 0, 0, 0, j.cap_max, KMER_MAX_K, 0, 0});
            auto& c = w.classes.back();
            c.count++;
            c.max_p1 = std::max(c.max_p1, j.g.p1);
            c.max_p2 = std::max(c.max_p2, j.g.p2);
            c.min_k = std::min(c.min_k, j.g.k);
        }
        TRY(capture_wave(b, w));
    }
    b->st.jobs = n_jobs;
    b->st.waves = (uint32_t)b->waves.size();
    return KMER_OK;
}

int create_batch(const kmer_batch_job* jobs, uint32_t n_jobs, uint64_t memory_budget, cudaStream_t stream,
                 kmer_batch** out) {
    auto* b = new (std::nothrow) kmer_batch;
    if (!b) return fail(KMER_ERR_OOM, "host allocation failed");
    std::unique_ptr<kmer_batch, void (*)(kmer_batch*)> guard(b, destroy_batch);
    CK(cudaGetDevice(&b->device));
    int smem_sm = 0, smem_optin = 0;
    CK(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device));
    CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, b->device));
    CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    b->leaf_budget = std::min<size_t>((size_t)smem_optin, (size_t)smem_sm / 2 - 1024 - 256);
    if (stream) {
        b->stream = stream;
    } else {
        CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
        CK(cudaDeviceSynchronize());  // readsets packed on the default stream are complete
    }
    prepare_pool(b->device);
    StreamScope scope(b->stream);
    b->jobs.resize(n_jobs);
    for (uint32_t i = 0; i < n_jobs; ++i) {
        BJob& j = b->jobs[i];
        j.rs = jobs[i].readset;
        j.p = jobs[i].params;
        j.survivors_hint = jobs[i].survivors_hint;
    }
    b->budget = memory_budget ? memory_budget : (size_t)(0.6 * (double)free_device_bytes());
    TRY(build_plan(b));
    guard.release();
    *out = b;
    return KMER_OK;
}

int run_alone(kmer_batch* b, BJob& j) {
    if (!j.alone) {
        kmer_analysis_params p = j.p;
        TRY(kmer_analysis_create(&p, b->stream, &j.alone));
    } else {
        TRY(kmer_analysis_reset(j.alone));
    }
    TRY(kmer_analysis_submit(j.alone, j.rs));
    TRY(kmer_analysis_query(j.alone, &j.alone_view));
    j.used_alone = true;
    j.n_out = j.alone_view.n;
    j.res_windows = j.alone_view.windows;
    j.res_distinct = j.alone_view.distinct;
    return KMER_OK;
}

// Leaves of job j that the wave's leaf kernel handed to the HBM recount
// (too many distinct keys or records for a shared-memory table): recounted
// now, while the wave's scratch still holds their records.  Returns false if
// the job must instead run alone (output too small for the extra survivors).
// Grows job j's output to `cap` survivors, keeping the first `keep`, and
// points its descriptor (host copy and the wave's device copy) at the new
// buffers.
int grow_output(kmer_batch* b, BJob& j, unsigned long long cap, unsigned long long keep) {
    if (cap <= j.out_cap) return KMER_OK;
    DevBuf nk, nc, ne, ncl;
    TRY(nk.ensure(cap * 8 * j.W + 16));
    TRY(nc.ensure(cap * 4 + 16));
    TRY(ne.ensure(cap * 32 + 16));
    TRY(ncl.ensure(cap * 2 + 16));
    if (keep) {
        CK(cudaMemcpyAsync(nk.p, j.out_keys.p, keep * 8 * j.W, cudaMemcpyDeviceToDevice, b->stream));
        CK(cudaMemcpyAsync(nc.p, j.out_count.p, keep * 4, cudaMemcpyDeviceToDevice, b->stream));
        CK(cudaMemcpyAsync(ne.p, j.out_ext.p, keep * 32, cudaMemcpyDeviceToDevice, b->stream));
        CK(cudaMemcpyAsync(ncl.p, j.out_cls.p, keep * 2, cudaMemcpyDeviceToDevice, b->stream));
    }
    j.out_keys = std::move(nk);
    j.out_count = std::move(nc);
    j.out_ext = std::move(ne);
    j.out_cls = std::move(ncl);
    j.out_cap = cap;
    j.job.out_keys = j.out_keys.as<unsigned long long>();
    j.job.out_count = j.out_count.as<unsigned>();
    j.job.out_ext = j.out_ext.as<unsigned>();
    j.job.out_cls = j.out_cls.as<unsigned char>();
    j.job.out_cap = cap;
    return KMER_OK;
}

int upload_desc(kmer_batch* b, BJob& j) {
    Wave& w = b->waves[j.wave];
    CK(cudaMemcpyAsync(w.d_jobs.as<Job>() + j.slot, &j.job, sizeof(Job), cudaMemcpyHostToDevice, b->stream));
    return KMER_OK;
}

// Repairs job j after its wave reported an undersized output, fallback list
// or level-2 layout: grows what was too small and re-runs, for this job
// alone, the stages after the scatter (the level-1 records are intact).
// *m is replaced by the job's counters after the re-run.
int repair_job(kmer_batch* b, BJob& j, unsigned idx, Misc* m) {
    const unsigned P = 1u << (j.g.p1 + j.g.p2);
    const bool relayout = j.g.p2 && (m->status & (ST_L2_OVERFLOW | ST_L2_PLAN));
    if (relayout) {
        // every record was counted toward its leaf even when it did not fit
        std::vector<unsigned long long> fill(P), exact(P + 1, 0);
        CK(cudaMemcpyAsync(fill.data(), j.job.l2_fill, P * 8ull, cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        for (unsigned i = 0; i < P; ++i) exact[i + 1] = exact[i] + fill[i];
        if (exact[P] > j.l2_capacity) return fail(KMER_ERR_TABLE_FULL, "level-2 records exceed the job's region");
        TRY(j.l2_exact.ensure((P + 1) * 8ull));
        CK(cudaMemcpyAsync(j.l2_exact.p, exact.data(), (P + 1) * 8ull, cudaMemcpyHostToDevice, b->stream));
        j.job.l2_leaf_start = j.l2_exact.as<unsigned long long>();
        j.job.l2_capacity = ~0ull;
        j.exact_p1 = j.g.p1;
        j.exact_p2 = j.g.p2;
    }
    if (m->status & ST_OUT_OVERFLOW) {
        // without dropped records out_n is the exact survivor count
        const unsigned long long want = relayout ? 2 * j.out_cap : m->out_n + m->out_n / 8 + 4096;
        TRY(grow_output(b, j, std::min<unsigned long long>(want, j.windows / j.p.min_count + 1024), 0));
    }
    if (m->status & ST_FALLBACK_FULL) {
        j.fb_cap = m->fb_n + 64;
        TRY(j.fb.ensure(j.fb_cap * 4ull));
        j.job.fb_list = j.fb.as<unsigned>();
        j.job.fb_cap = j.fb_cap;
    }
    TRY(upload_desc(b, j));
    // fresh counters, keeping the windows the scatter emitted
    Misc z{};
    z.stats[2] = m->stats[2];
    CK(cudaMemcpyAsync(b->misc.as<Misc>() + idx, &z, sizeof z, cudaMemcpyHostToDevice, b->stream));
    Wave& w = b->waves[j.wave];
    const Job* dj = w.d_jobs.as<Job>() + j.slot;
    unsigned long long* maps = b->one_maps.as<unsigned long long>();
    const unsigned long long leaf_off[2] = {0ull, (unsigned long long)P};
    CK(cudaMemcpyAsync(maps, leaf_off, 16, cudaMemcpyHostToDevice, b->stream));
    if (relayout) {
        CK(cudaMemsetAsync(j.job.l2_fill, 0, P * 8ull, b->stream));
        CK(launch_l2_plan(dj, 1, maps + 2, b->stream));
        CK(launch_repart(j.W, dj, maps + 2, 1, j.g.p2, b->num_sms, b->stream));
    }
    CK(launch_leaf(j.W, dj, maps, 1, P, j.cap_max, b->num_sms, b->stream));
    CK(launch_leaf_split(j.W, dj, 1, j.cap_max, b->num_sms, b->stream));
    CK(cudaMemcpyAsync(&b->host_misc[idx], b->misc.as<Misc>() + idx, sizeof(Misc), cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    *m = b->host_misc[idx];
    return KMER_OK;
}

int batch_fallbacks(kmer_batch* b, BJob& j, unsigned idx, const Misc& m, bool* ok) {
    *ok = false;
    const unsigned n = m.fb_n;
    std::vector<unsigned> leaves(n);
    CK(cudaMemcpyAsync(leaves.data(), j.fb.as<unsigned>(), n * 4ull, cudaMemcpyDeviceToHost, b->stream));
    std::vector<unsigned long long> fill(n);
    const unsigned long long* fsrc = j.g.p2 ? j.job.l2_fill : j.job.l1_fill;
    CK(cudaStreamSynchronize(b->stream));
    for (unsigned i = 0; i < n; ++i)  // a range's records are at most its leaf's
        CK(cudaMemcpyAsync(&fill[i], fsrc + fallback_leaf(leaves[i]), 8, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    unsigned long long extra = 0, max_n = 0;
    for (unsigned i = 0; i < n; ++i) {
        extra += fill[i] / j.p.min_count + 1;
        max_n = std::max(max_n, fill[i]);
    }
    if (m.out_n + extra > j.out_cap) {  // room for the recounted leaves' survivors
        TRY(grow_output(b, j, m.out_n + extra + (m.out_n + extra) / 8 + 4096, m.out_n));
        TRY(upload_desc(b, j));
    }
    const size_t eb = hbm_entry_bytes(j.W);
    TRY(b->hbm.ensure(next_pow2(std::max<unsigned long long>(1024, 2 * max_n)) * eb));
    for (unsigned i = 0; i < n; ++i) {
        const unsigned long long c = next_pow2(std::max<unsigned long long>(1024, 2 * fill[i]));
        CK(cudaMemsetAsync(b->hbm.p, 0, c * eb, b->stream));
        CK(launch_records_insert(j.job, leaves[i], b->hbm.p, c, b->num_sms, b->stream));
        CK(launch_hbm_sweep(j.job, b->hbm.p, c, b->num_sms, b->stream));
    }
    Misc after{};
    CK(cudaMemcpyAsync(&after, b->misc.as<Misc>() + idx, sizeof(Misc), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    b->host_misc[idx] = after;
    *ok = after.status == 0 && after.stats[0] == after.stats[2];
    b->st.fallback_leaves += n;
    return KMER_OK;
}

int run_batch(kmer_batch* b) {
    const auto t0 = std::chrono::steady_clock::now();
    StreamScope scope(b->stream);
    b->have_result = false;
    b->st.graph_launches = 0;
    b->st.jobs_alone = 0;
    b->st.fallback_leaves = 0;
    b->st.jobs_repaired = 0;
    b->st.alone_level1 = 0;
    b->st.alone_other = 0;
    if (b->replan) {  // sizing learned from the previous run
        TRY(build_plan(b));
        b->replan = false;
        b->st.replans++;
    }
    if (b->own_stream) CK(cudaDeviceSynchronize());  // re-packed readsets on other streams are complete
    const size_t n = b->jobs.size();
    std::vector<char> good(n, 0);
    for (auto& w : b->waves) {
        CK(cudaGraphLaunch(w.exec, b->stream));
        b->st.graph_launches++;
        // check the wave before the next one reuses its scratch
        CK(cudaMemcpyAsync(b->host_misc.data(), b->misc.p, n * sizeof(Misc), cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        for (unsigned id : w.ids) {
            Misc m = b->host_misc[id];
            BJob& j = b->jobs[id];
            const unsigned repairable = ST_L2_OVERFLOW | ST_L2_PLAN | ST_OUT_OVERFLOW | ST_FALLBACK_FULL;
            bool repaired = false;
            for (int attempt = 0; attempt < 3 && m.status && !(m.status & ~repairable); ++attempt) {
                TRY(repair_job(b, j, id, &m));
                repaired = true;
            }
            if (repaired) b->st.jobs_repaired++;
            if (m.status == 0 && m.fb_n == 0 && m.stats[0] == m.stats[2]) {
                good[id] = 1;
            } else if (m.status == 0 && m.fb_n > 0) {
                bool ok = false;
                TRY(batch_fallbacks(b, j, id, m, &ok));
                good[id] = ok ? 1 : 0;
            }
            if (!good[id]) {
                if (m.status & ST_L1_OVERFLOW) b->st.alone_level1++;
                else b->st.alone_other++;
            }
        }
    }
    for (size_t i = 0; i < n; ++i) {
        BJob& j = b->jobs[i];
        j.used_alone = false;
        if (j.windows == 0) {
            j.n_out = j.res_windows = j.res_distinct = 0;
            continue;
        }
        if (good[i]) {
            const Misc& m = b->host_misc[i];
            j.n_out = m.out_n;
            j.res_windows = m.stats[0];
            j.res_distinct = m.stats[1];
        } else {  // level-1 overflow, failed wait or too large for a wave: exact regular path
            if (j.wave < 0) b->st.alone_other++;
            TRY(run_alone(b, j));
            b->st.jobs_alone++;
        }
    }
    // sizing for the next run: a job whose distinct keys were far from what its
    // geometry was planned for gets its counts as hints (its leaves keep the
    // planned number of keys each), and the batch is re-planned before that run
    for (size_t i = 0; i < n; ++i) {
        BJob& j = b->jobs[i];
        // a job with a learned exact leaf layout keeps its plan
        if (j.windows == 0 || j.used_alone || !good[i] || j.l2_exact.p) continue;
        const double r = (double)j.res_distinct / (double)j.basis;
        if (r > 1.1 || r < 0.75) {
            if (j.p.leaf_bits) {
                const double per_leaf = (double)j.basis / (double)(1ull << j.p.leaf_bits);
                unsigned lb = ceil_log2((unsigned long long)std::max(2.0, (double)j.res_distinct / per_leaf));
                j.p.leaf_bits = std::min(22u, std::max(1u, lb));
                j.p.l1_bits = 0;
            }
            j.p.distinct_hint = j.res_distinct + j.res_distinct / 16 + 1;
            j.survivors_hint = j.n_out;
            b->replan = true;
        }
    }
    b->st.ms_total = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    b->have_result = true;
    return KMER_OK;
}

}  // namespace

extern "C" {

int kmer_batch_create(const kmer_batch_job* jobs, uint32_t n_jobs, uint64_t memory_budget, void* cuda_stream,
                      kmer_batch_t** out) {
    if (!out) return fail(KMER_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_jobs && !jobs) return fail(KMER_ERR_INVALID_ARG, "jobs is NULL");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(KMER_ERR_NO_DEVICE, "no CUDA device");
    }
    for (uint32_t i = 0; i < n_jobs; ++i) {
        const kmer_analysis_params& p = jobs[i].params;
        if (!jobs[i].readset) return fail(KMER_ERR_INVALID_ARG, "job %u has no readset", i);
        if (p.k == 0 || p.k > KMER_MAX_K || p.k % 2 == 0 || p.min_count == 0 || p.ext_mode > 1 ||
            (p.ext_mode == 0 && p.err_den == 0) || p.variant != KMER_VARIANT_PARTITIONED || p.leaf_bits > 22 ||
            p.l1_bits > 11)
            return fail(KMER_ERR_INVALID_ARG, "job %u has invalid parameters", i);
        if (jobs[i].readset->qual_offset != p.qual_offset || jobs[i].readset->qual_threshold != p.qual_threshold)
            return fail(KMER_ERR_INVALID_ARG, "job %u: readset packed with other quality parameters", i);
        if (jobs[i].readset->device != dev) return fail(KMER_ERR_INVALID_ARG, "job %u: readset on another device", i);
    }
    return create_batch(jobs, n_jobs, memory_budget, static_cast<cudaStream_t>(cuda_stream), out);
}

int kmer_batch_run(kmer_batch_t* b) {
    if (!b) return fail(KMER_ERR_INVALID_ARG, "NULL batch");
    return run_batch(b);
}

int kmer_batch_result(kmer_batch_t* b, uint32_t job, kmer_result_view* out) {
    if (!b || !out) return fail(KMER_ERR_INVALID_ARG, "NULL batch or output");
    if (job >= b->jobs.size()) return fail(KMER_ERR_INVALID_ARG, "job %u out of range", job);
    if (!b->have_result) return fail(KMER_ERR_BAD_STATE, "batch has not run");
    BJob& j = b->jobs[job];
    std::memset(out, 0, sizeof *out);
    if (j.used_alone) {
        *out = j.alone_view;
        return KMER_OK;
    }
    out->n = j.n_out;
    out->k = j.p.k;
    out->words = j.W;
    out->keys = j.out_keys.as<uint64_t>();
    out->count = j.out_count.as<uint32_t>();
    out->ext = j.out_ext.as<uint32_t>();
    out->cls = j.out_cls.as<uint8_t>();
    out->windows = j.res_windows;
    out->distinct = j.res_distinct;
    return KMER_OK;
}

int kmer_batch_copy_results(kmer_batch_t* b, uint32_t job, uint64_t* keys, uint32_t* count, uint32_t* ext,
                            uint8_t* cls, uint64_t capacity) {
    kmer_result_view v;
    TRY(kmer_batch_result(b, job, &v));
    if (capacity < v.n) return fail(KMER_ERR_INVALID_ARG, "capacity %llu < %llu results",
                                    (unsigned long long)capacity, (unsigned long long)v.n);
    if (v.n) {
        if (keys) CK(cudaMemcpyAsync(keys, v.keys, v.n * 8 * v.words, cudaMemcpyDeviceToHost, b->stream));
        if (count) CK(cudaMemcpyAsync(count, v.count, v.n * 4, cudaMemcpyDeviceToHost, b->stream));
        if (ext) CK(cudaMemcpyAsync(ext, v.ext, v.n * 32, cudaMemcpyDeviceToHost, b->stream));
        if (cls) CK(cudaMemcpyAsync(cls, v.cls, v.n * 2, cudaMemcpyDeviceToHost, b->stream));
    }
    CK(cudaStreamSynchronize(b->stream));
    return KMER_OK;
}

int kmer_batch_get_stats(const kmer_batch_t* b, kmer_batch_stats* out) {
    if (!b || !out) return fail(KMER_ERR_INVALID_ARG, "NULL batch or output");
    *out = b->st;
    return KMER_OK;
}

int kmer_batch_destroy(kmer_batch_t* b) {
    if (!b) return KMER_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    StreamScope scope(b->stream);
    destroy_batch(b);
    return KMER_OK;
}

}  // extern "C"
