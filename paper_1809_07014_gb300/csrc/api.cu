// Host side of the C ABI declared in include/kmer_analysis.h: readsets,
// planning (passes, partition bits, buffer sizes), launches, the retry loop
// that grows any buffer a device kernel found too small, and the HBM-table
// fallback for partitions that do not fit on chip.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "kmer_analysis.h"

using namespace kmer;

#include "host.h"

namespace kmer {
namespace {
thread_local std::string g_err;
}  // namespace

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

const char* last_error_message() { return g_err.c_str(); }

thread_local cudaStream_t tl_alloc_stream = nullptr;

void prepare_pool(int device) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), device) != done.end()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        unsigned long long keep = ~0ull;  // freed memory stays in the pool for reuse
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.push_back(device);
}

size_t free_device_bytes() {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int dev = 0;
    cudaMemPool_t pool;
    unsigned long long reserved = 0, used = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
        fr += (size_t)(reserved - used);
    cudaGetLastError();
    return fr;
}

namespace {
struct PinnedMiscPool {
    std::mutex mu;
    std::vector<Misc*> free_list;
};
PinnedMiscPool& pinned_pool() {
    static PinnedMiscPool* pool = new PinnedMiscPool;  // lives for the whole process
    return *pool;
}
}  // namespace

Misc* pinned_misc_get() {
    PinnedMiscPool& pool = pinned_pool();
    std::lock_guard<std::mutex> lk(pool.mu);
    if (pool.free_list.empty()) {
        constexpr int kChunk = 64;  // Misc blocks per pinned allocation (never returned)
        Misc* chunk = nullptr;
        if (cudaMallocHost((void**)&chunk, kChunk * sizeof(Misc)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int i = kChunk - 1; i >= 0; --i) pool.free_list.push_back(chunk + i);
    }
    Misc* m = pool.free_list.back();
    pool.free_list.pop_back();
    return m;
}

void pinned_misc_put(Misc* m) {
    if (!m) return;
    PinnedMiscPool& pool = pinned_pool();
    std::lock_guard<std::mutex> lk(pool.mu);
    pool.free_list.push_back(m);
}

Geometry plan_geometry(unsigned k, unsigned long long windows, unsigned long long basis, size_t budget,
                       unsigned cap_max, unsigned leaf_bits, unsigned l1_bits, bool waves, double l1_slack) {
    Geometry g{};
    g.k = k;
    g.W = (2 * k + 63) / 64;
    g.hb = 2 * k - 64 * (g.W - 1);
    g.bt = g.W == 1 ? 2 * k : 64;
    // up to 0.7 of a leaf table of (estimated) distinct keys per leaf: the
    // estimate carries a 15 % margin, so leaves hold about 0.3-0.6 of a table
    // (fewer, fuller leaves amortise each leaf's sweep and barriers; a leaf
    // that overflows is counted again in key ranges)
    const unsigned long long target = std::max(64ull, (unsigned long long)cap_max * 7 / 10);
    unsigned p = leaf_bits ? leaf_bits : ceil_log2((basis + target - 1) / target);
    const unsigned need = g.bt > 58 ? g.bt - 58 : 0;  // partition bits implied by the record format
    p = std::max(p, need);
    p = std::min(p, g.bt);
    // passes: records of one pass (two levels, with slack) must fit the budget;
    // with level-2 waves, the level-1 records and one wave of the level 2
    const double rec_bytes = 8.0 * g.W;
    unsigned ps = 0;
    for (;;) {
        const double win = (double)windows / (double)(1ull << ps);
        const double bytes = win * rec_bytes * (waves ? 1.0 + l1_slack + 2.1 / kMaxWaves : 3.5) +
                             64.0 * (double)(1ull << (p > ps ? p - ps : 0)) * 8;
        if (bytes <= (waves ? 0.9 : 0.8) * (double)budget || ps >= p || ps >= 12) break;
        ++ps;
    }
    const unsigned lb = p - ps;
    unsigned p1, p2;
    if (lb <= 11) {
        p1 = lb;
        p2 = 0;
    } else {
        // the scatter's cost grows with its fan-out more than the repartition's does
        p1 = std::min(11u, lb / 2);
        if (l1_bits >= 1 && l1_bits <= 11 && l1_bits < lb) p1 = l1_bits;
        p2 = lb - p1;
        if (p2 > 11) p2 = 11;
    }
    if (ps + p1 < need) p1 = need - ps;
    g.ps = ps;
    g.p1 = p1;
    g.p2 = p2;
    return g;
}

}  // namespace kmer

using namespace kmer;


struct kmer_analysis {
    kmer_analysis_params p{};
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    size_t leaf_smem_budget = 0;
    std::vector<const kmer_readset*> submitted;
    std::vector<kmer_readset*> owned;
    // device buffers
    DevBuf l1_rec, l1_start, l1_cap, l1_fill;
    DevBuf l2_rec, l2_base, l2_leafcap, l2_fill, l2_leaf_start, tile_prefix;
    DevBuf out_keys, out_count, out_ext, out_cls;
    DevBuf fb_list, split_list, hbm, misc;
    DevBuf gate1, gate2, gate_cnt;  // Bloom gate: filters F1, F2 and the gate pass's counters
    DevBuf trav_scratch, trav_bases, trav_off, trav_tot;  // graph traversal: scratch and contigs
    DevBuf sort_buf;  // sorted output: scratch when no records buffer is large enough
    unsigned long long n_contigs = 0, contig_bases = 0;
    bool have_contigs = false;
    DevBuf lk_index, lk_keys, lk_out;  // survivors' index for lookups, staging of host lookups
    // survivors written straight into caller buffers (kmer_analysis_query_into): device
    // addresses of those buffers while such a query runs, and of the results after it
    bool ext_out = false;
    unsigned long long* res_keys = nullptr;
    unsigned* res_count = nullptr;
    unsigned* res_ext = nullptr;
    unsigned char* res_cls = nullptr;
    unsigned long long lk_cap = 0;     // index slots; 0 = no index for the current results
    DevBuf d_ajob, d_sjobs, d_tile_off, d_leaf_off, d_job_tile_off;  // job descriptors and work maps
    unsigned long long out_cap = 0, fb_cap = 0;
    Misc* host_misc = nullptr;  // pinned
    // profiling (KMER_FLAG_PROFILE): one begin/end event pair per stage
    enum { STG_SCATTER, STG_REPART, STG_LEAF, STG_FALLBACK, STG_GATE, STG_SORT, STG_N };
    cudaEvent_t ev_b[STG_N] = {}, ev_e[STG_N] = {};
    bool ev_pending[STG_N] = {};
    // results
    bool have_result = false;
    unsigned long long n_out = 0, res_windows = 0, res_distinct = 0;
    unsigned long long out_hint = 0;  // survivors of the previous query (buffer sizing)
    // sizing learned from earlier queries: distinct / windows at this k, and the
    // level-2 leaf slack (grown whenever a leaf overflowed)
    unsigned hist_k = 0;
    double hist_ratio = 0.0;
    unsigned l2_slack_num = 512;  // leaf capacity = 2 * mean + 256
    double hint_ratio = 0.0;      // distinct_hint / windows of the current query (0 = no hint)
    // Bloom gate: filter words (log2), and first sightings / windows at hist_k
    unsigned gate_bits = 0;
    double gate_ratio = 0.0;
    // level-1 buckets of the last large single-pass query at l1_imb_k: a high
    // quantile of the fills over the mean, and every bucket's fill (for buckets
    // far above the rest, such as one holding a heavy hitter)
    unsigned l1_imb_k = 0, l1_prev_p1 = 0;
    double l1_imbalance = 0.0;
    std::vector<unsigned long long> l1_prev_fill;
    unsigned long long l1_prev_windows = 0;
    kmer_analysis_stats st{};

    unsigned W() const { return (2 * p.k + 63) / 64; }
    size_t device_bytes() const {
        const DevBuf* bs[] = {&l1_rec, &l1_start, &l1_cap, &l1_fill, &l2_rec, &l2_base, &l2_leafcap, &l2_fill,
                              &l2_leaf_start, &tile_prefix, &out_keys, &out_count, &out_ext, &out_cls,
                              &fb_list, &split_list, &hbm, &misc, &lk_index, &lk_keys, &lk_out, &d_ajob,
                              &d_sjobs, &d_tile_off, &d_leaf_off,
                              &d_job_tile_off, &gate1, &gate2, &gate_cnt, &trav_scratch, &trav_bases, &trav_off,
                              &trav_tot, &sort_buf};
        size_t t = 0;
        for (auto* b : bs) t += b->bytes;
        return t;
    }
};

namespace {

int validate_params(const kmer_analysis_params* p) {
    if (!p) return fail(KMER_ERR_INVALID_ARG, "params is NULL");
    if (p->k == 0 || p->k > KMER_MAX_K || p->k % 2 == 0)
        return fail(KMER_ERR_INVALID_ARG, "k must be odd and in 1..%d (got %u)", KMER_MAX_K, p->k);
    if (p->min_count == 0) return fail(KMER_ERR_INVALID_ARG, "min_count must be >= 1");
    if (p->ext_mode > 1) return fail(KMER_ERR_INVALID_ARG, "unknown ext_mode %u", p->ext_mode);
    if (p->ext_mode == 0 && p->err_den == 0) return fail(KMER_ERR_INVALID_ARG, "err_den must be > 0");
    if (p->variant > 1) return fail(KMER_ERR_INVALID_ARG, "unknown variant %u", p->variant);
    if (p->qual_offset > 255 || p->qual_threshold > 255)
        return fail(KMER_ERR_INVALID_ARG, "qual_offset and qual_threshold must fit a byte");
    if (p->leaf_bits > 22) return fail(KMER_ERR_INVALID_ARG, "leaf_bits must be <= 22");
    if (p->l1_bits > 11) return fail(KMER_ERR_INVALID_ARG, "l1_bits must be <= 11");
    if (p->flags & ~(KMER_FLAG_PROFILE | KMER_FLAG_BLOOM_GATE | KMER_FLAG_SORTED_OUTPUT))
        return fail(KMER_ERR_INVALID_ARG, "unknown flags 0x%x", p->flags);
    if ((p->flags & KMER_FLAG_BLOOM_GATE) && p->min_count < 2)
        return fail(KMER_ERR_INVALID_ARG, "the Bloom gate needs min_count >= 2 (it drops k-mers seen once)");
    if ((p->flags & KMER_FLAG_BLOOM_GATE) && p->variant != KMER_VARIANT_PARTITIONED)
        return fail(KMER_ERR_INVALID_ARG, "the Bloom gate works with the partitioned variant only");
    for (unsigned r : p->reserved)
        if (r) return fail(KMER_ERR_INVALID_ARG, "reserved fields must be zero");
    return KMER_OK;
}

bool valid_where(int where) { return where == KMER_HOST || where == KMER_DEVICE || where == KMER_HOST_STAGED; }

// Device address of page-locked host memory, or null for any other pointer.
const void* host_mapped(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// A large host<->device copy in pieces (64 MB, at most two in flight; the
// calling thread waits).  Copies in one direction share a copy engine in
// submission order: a small copy that another stream submits (counters,
// descriptors) then waits for one piece, not for the whole transfer.
#ifndef KMER_COPY_PIECE_MB
#define KMER_COPY_PIECE_MB 64
#endif
#ifndef KMER_COPY_INFLIGHT
#define KMER_COPY_INFLIGHT 2
#endif
cudaError_t paced_copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    constexpr size_t kPiece = (size_t)KMER_COPY_PIECE_MB << 20;
    constexpr unsigned kInFlight = KMER_COPY_INFLIGHT;
    if (bytes <= kInFlight * kPiece) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    cudaEvent_t ev[kInFlight] = {};
    cudaError_t e = cudaSuccess;
    for (unsigned i = 0; i < kInFlight && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    for (size_t off = 0, k = 0; e == cudaSuccess && off < bytes; off += kPiece, ++k) {
        if (k >= kInFlight) e = cudaEventSynchronize(ev[k % kInFlight]);
        if (e != cudaSuccess) break;
        const size_t n = bytes - off < kPiece ? bytes - off : kPiece;
        e = cudaMemcpyAsync(static_cast<char*>(dst) + off, static_cast<const char*>(src) + off, n, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[k % kInFlight], s);
    }
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    return e;
}

int pack_readset(kmer_readset* rs, const char* bases, const uint8_t* quals, const uint64_t* offsets,
                 uint64_t n_reads, int where, cudaStream_t s) {
    rs->n_reads = 0;
    rs->n_bases = 0;
    rs->n_blocks = 0;
    rs->launches = 0;
    std::memset(rs->len_stats, 0, sizeof rs->len_stats);
    if (n_reads == 0) return KMER_OK;
    const char* d_bases = bases;
    const uint8_t* d_quals = quals;
    TRY(rs->offsets.ensure((n_reads + 1) * 8));
    if (where != KMER_DEVICE) {
        // offsets are checked on the device (read_geometry_kernel)
        CK(cudaMemcpyAsync(rs->offsets.p, offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice, s));
        // page-locked host memory is read in place by the pack kernel over the
        // host link (one pass, no staging copy) unless staging is asked for;
        // other host memory is staged
        const bool in_place = where == KMER_HOST;
        const char* mb = in_place ? static_cast<const char*>(host_mapped(bases)) : nullptr;
        const uint8_t* mq = in_place ? static_cast<const uint8_t*>(host_mapped(quals)) : nullptr;
        if (mb && mq) {
            d_bases = mb;
            d_quals = mq;
        } else {
            const unsigned long long nb = offsets[n_reads];
            TRY(rs->tmp_bases.ensure(nb + 16));
            TRY(rs->tmp_quals.ensure(nb + 16));
            CK(paced_copy(rs->tmp_bases.p, bases, nb, s));
            CK(paced_copy(rs->tmp_quals.p, quals, nb, s));
            d_bases = rs->tmp_bases.as<char>();
            d_quals = rs->tmp_quals.as<uint8_t>();
        }
    } else {
        CK(cudaMemcpyAsync(rs->offsets.p, offsets, (n_reads + 1) * 8, cudaMemcpyDeviceToDevice, s));
    }
    const unsigned long long* d_off = rs->offsets.as<unsigned long long>();
    // read geometry: blocks per read, length histogram, monotonicity
    TRY(rs->nblk.ensure(n_reads * 8));
    TRY(rs->blk_off.ensure((n_reads + 1) * 8));
    TRY(rs->scratch.ensure(scan_temp_bytes(n_reads)));
    const size_t stats_bytes = (kLenHist + 2) * 8;
    TRY(rs->stats.ensure(stats_bytes + 3 * 8));
    CK(cudaMemsetAsync(rs->stats.p, 0, stats_bytes, s));
    unsigned long long* st = rs->stats.as<unsigned long long>();
    unsigned int* bad = reinterpret_cast<unsigned int*>(st + kLenHist);
    CK(launch_read_geometry(d_off, n_reads, rs->nblk.as<unsigned long long>(), st, bad, s));
    CK(exclusive_scan_u64(rs->nblk.as<unsigned long long>(), rs->blk_off.as<unsigned long long>(), n_reads,
                          rs->scratch.p, s));
    // gather the totals next to the histogram so that one copy brings everything back
    CK(cudaMemcpyAsync(st + kLenHist + 2, rs->blk_off.as<unsigned long long>() + n_reads, 8,
                       cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(st + kLenHist + 3, d_off, 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(st + kLenHist + 4, d_off + n_reads, 8, cudaMemcpyDeviceToDevice, s));
    std::vector<unsigned long long> host(kLenHist + 5);
    CK(cudaMemcpyAsync(host.data(), st, host.size() * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const unsigned bad_flags = (unsigned)(host[kLenHist] & 0xFFFFFFFFull);
    if (bad_flags & 1u) return fail(KMER_ERR_INVALID_ARG, "offsets are not non-decreasing");
    if (bad_flags & 2u) return fail(KMER_ERR_INVALID_ARG, "a read is 2^31 bases or longer");
    const unsigned long long total_blocks = host[kLenHist + 2];
    TRY(rs->blocks.ensure(std::max<unsigned long long>(total_blocks, 1) * sizeof(PackedBlock)));
    int num_sms = 0;
    CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, rs->device));
    CK(launch_pack(d_bases, d_quals, d_off, rs->blk_off.as<unsigned long long>(), n_reads, rs->qual_offset,
                   rs->qual_threshold, rs->blocks.as<PackedBlock>(), num_sms, s));
    CK(cudaStreamSynchronize(s));
    std::memcpy(rs->len_stats, host.data(), sizeof(rs->len_stats));
    rs->n_blocks = total_blocks;
    rs->n_bases = host[kLenHist + 4] - host[kLenHist + 3];
    rs->n_reads = n_reads;
    rs->launches = 5;  // geometry, three scan phases, pack
    return KMER_OK;
}

// The caller has made sure no stream still reads the readset; its buffers
// are freed in the order of the legacy stream, which always exists (the
// streams they were packed on may be gone).
void destroy_readset(kmer_readset* rs) {
    DevBuf* bs[] = {&rs->blocks, &rs->blk_off, &rs->offsets, &rs->tmp_bases, &rs->tmp_quals,
                    &rs->nblk, &rs->scratch, &rs->stats};
    for (auto* b : bs) {
        b->s = nullptr;
        b->release();
    }
    delete rs;
}

int make_readset(const char* bases, const uint8_t* quals, const uint64_t* offsets, uint64_t n_reads,
                 uint32_t qual_offset, uint32_t qual_threshold, int where, cudaStream_t s, kmer_readset** out) {
    if (!out) return fail(KMER_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_where(where)) return fail(KMER_ERR_INVALID_ARG, "where must be HOST, DEVICE or HOST_STAGED");
    if (n_reads && (!bases || !quals || !offsets))
        return fail(KMER_ERR_INVALID_ARG, "bases, quals and offsets must be non-NULL when n_reads > 0");
    if (qual_offset > 255 || qual_threshold > 255)
        return fail(KMER_ERR_INVALID_ARG, "qual_offset and qual_threshold must fit a byte");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(KMER_ERR_NO_DEVICE, "no CUDA device");
    }
    auto* rs = new (std::nothrow) kmer_readset;
    if (!rs) return fail(KMER_ERR_OOM, "host allocation failed");
    rs->device = dev;
    prepare_pool(dev);
    StreamScope scope(s);
    rs->qual_offset = qual_offset;
    rs->qual_threshold = qual_threshold;
    int rc = pack_readset(rs, bases, quals, offsets, n_reads, where, s);
    if (rc != KMER_OK) {
        cudaStreamSynchronize(s);  // nothing may still use the buffers
        cudaGetLastError();
        destroy_readset(rs);
        return rc;
    }
    // a one-shot readset keeps only its packed form; kmer_readset_pack keeps staging for reuse
    rs->tmp_bases.release();
    rs->tmp_quals.release();
    rs->nblk.release();
    rs->scratch.release();
    *out = rs;
    return KMER_OK;
}


// ------------------------------------------------------------------ planning
struct Plan {
    Geometry g;
    unsigned passes;
    unsigned long long windows;  // upper bound (N windows included)
    size_t budget;               // device bytes for the records of a pass
};

// Level-1 slack: an eighth of a bucket's mean, or, after a large query at the
// same k, a quarter more than the largest bucket's excess over the mean then
// (repeated k-mers make bucket sizes vary far more than a uniform spread).
double l1_slack(const kmer_analysis* h) {
    if (h->l1_imb_k == h->p.k && h->l1_imbalance > 0.0)
        return std::min(0.25, std::max(0.02, (h->l1_imbalance - 1.0) * 1.25 + 0.01));
    return 0.125;
}

Plan make_plan(const kmer_analysis* h, unsigned long long windows, size_t budget, unsigned cap_max,
               unsigned long long gated_distinct = 0) {
    Plan pl{};
    pl.windows = windows;
    unsigned long long basis = windows;
    if (gated_distinct) basis = std::min<unsigned long long>(windows, gated_distinct + gated_distinct / 8 + 1024);
    else if (h->p.distinct_hint) basis = std::min<unsigned long long>(h->p.distinct_hint, windows);
    else if (h->hist_k == h->p.k && h->hist_ratio > 0.0)  // learned from the previous query at this k
        basis = std::min<unsigned long long>(windows, (unsigned long long)(1.15 * h->hist_ratio * (double)windows) + 1);
    pl.g = plan_geometry(h->p.k, windows, basis, budget, cap_max, h->p.leaf_bits, h->p.l1_bits, true, l1_slack(h));
    pl.passes = 1u << pl.g.ps;
    pl.budget = budget;
    return pl;
}

int read_misc(kmer_analysis* h) {
    CK(cudaMemcpyAsync(h->host_misc, h->misc.p, sizeof(Misc), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return KMER_OK;
}

int ensure_output(kmer_analysis* h, unsigned long long cap, unsigned long long keep) {
    if (cap <= h->out_cap) return KMER_OK;
    if (h->ext_out)  // the caller's buffers cannot grow
        return fail(KMER_ERR_INVALID_ARG, "output capacity %llu < %llu survivors", h->out_cap, cap);
    const unsigned W = h->W();
    cap = std::max(cap, (unsigned long long)1024);
    DevBuf nk, nc, ne, ncl;
    TRY(nk.ensure(cap * 8 * W));
    TRY(nc.ensure(cap * 4));
    TRY(ne.ensure(cap * 32));
    TRY(ncl.ensure(cap * 2));
    if (keep) {
        CK(cudaMemcpyAsync(nk.p, h->out_keys.p, keep * 8 * W, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(nc.p, h->out_count.p, keep * 4, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(ne.p, h->out_ext.p, keep * 32, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(ncl.p, h->out_cls.p, keep * 2, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    std::swap(h->out_keys, nk);
    std::swap(h->out_count, nc);
    std::swap(h->out_ext, ne);
    std::swap(h->out_cls, ncl);
    nk.release();
    nc.release();
    ne.release();
    ncl.release();
    h->out_cap = cap;
    return KMER_OK;
}

// The results live in the analysis's own output buffers (after they may have moved).
void fill_job_outputs_ptrs(kmer_analysis* h) {
    h->res_keys = h->out_keys.as<unsigned long long>();
    h->res_count = h->out_count.as<unsigned int>();
    h->res_ext = h->out_ext.as<unsigned int>();
    h->res_cls = h->out_cls.as<unsigned char>();
}

void fill_job_outputs(kmer_analysis* h, Job& j) {
    Misc* m = h->misc.as<Misc>();
    if (!h->ext_out) {
        h->res_keys = h->out_keys.as<unsigned long long>();
        h->res_count = h->out_count.as<unsigned int>();
        h->res_ext = h->out_ext.as<unsigned int>();
        h->res_cls = h->out_cls.as<unsigned char>();
    }
    j.out_keys = h->res_keys;
    j.out_count = h->res_count;
    j.out_ext = h->res_ext;
    j.out_cls = h->res_cls;
    j.out_cap = h->out_cap;
    j.out_n = &m->out_n;
    j.status = &m->status;
    j.stats = m->stats;
    j.fb_list = h->fb_list.as<unsigned int>();
    j.fb_n = &m->fb_n;
    j.fb_cap = (unsigned)h->fb_cap;
    j.split_list = h->split_list.as<unsigned int>();
    j.split_n = &m->split_n;
    j.split_cap = (unsigned)(h->split_list.bytes / 4);
    j.min_count = h->p.min_count;
    j.ext_mode = h->p.ext_mode;
    j.t_base = h->p.t_base;
    j.err_num = h->p.err_num;
    j.err_den = h->p.err_den;
    j.t_ext = h->p.t_ext;
    j.l2_slack_num = h->l2_slack_num;
    // leaf table: twice the expected distinct keys of a leaf (one slot per record if unknown)
    double ratio = 1.0;
    if (h->hist_k == h->p.k && h->hist_ratio > 0.0) ratio = std::min(1.0, 2.0 * h->hist_ratio + 0.05);
    else if (h->hint_ratio > 0.0) ratio = std::min(1.0, 2.0 * h->hint_ratio + 0.05);
    j.table_ratio_num = (unsigned)(ratio * 65536.0);
}

void set_readset(Job& j, const kmer_readset* rs) {
    j.blocks = rs->blocks.as<PackedBlock>();
    j.blk_off = rs->blk_off.as<unsigned long long>();
    j.offsets = rs->offsets.as<unsigned long long>();
    j.n_reads = rs->n_reads;
}

// Copy a host array to a device buffer (pageable source: the call returns once
// the data is staged, so the host array may change right after).
template <class T>
int upload(kmer_analysis* h, DevBuf& dst, const std::vector<T>& src) {
    TRY(dst.ensure(std::max<size_t>(src.size() * sizeof(T), 16)));
    if (!src.empty()) CK(cudaMemcpyAsync(dst.p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    return KMER_OK;
}

// Reset the per-pass device counters; out_n restarts at `out_start` and the
// scatter's emitted-window count at `emitted` (kept when only later stages re-run).
int reset_misc(kmer_analysis* h, unsigned long long out_start, unsigned long long emitted = 0) {
    Misc m{};
    m.out_n = out_start;
    m.stats[2] = emitted;
    std::memcpy(h->host_misc, &m, sizeof m);
    CK(cudaMemcpyAsync(h->misc.p, h->host_misc, sizeof(Misc), cudaMemcpyHostToDevice, h->stream));
    return KMER_OK;
}

int status_error(unsigned st) {
    if (st & ST_TIMEOUT) return fail(KMER_ERR_TIMEOUT, "a bounded device wait gave up");
    if (st & ST_COUNTER_OVERFLOW) return fail(KMER_ERR_COUNTER_OVERFLOW, "a k-mer count exceeded 2^32-1");
    if (st & ST_TABLE_FULL) return fail(KMER_ERR_TABLE_FULL, "an HBM table ran out of slots");
    return KMER_OK;
}

bool profiling(const kmer_analysis* h) { return (h->p.flags & KMER_FLAG_PROFILE) != 0; }

int prof_begin(kmer_analysis* h, int stg) {
    if (!profiling(h)) return KMER_OK;
    if (!h->ev_b[stg]) {
        CK(cudaEventCreate(&h->ev_b[stg]));
        CK(cudaEventCreate(&h->ev_e[stg]));
    }
    CK(cudaEventRecord(h->ev_b[stg], h->stream));
    return KMER_OK;
}

int prof_end(kmer_analysis* h, int stg) {
    if (!profiling(h)) return KMER_OK;
    CK(cudaEventRecord(h->ev_e[stg], h->stream));
    h->ev_pending[stg] = true;
    return KMER_OK;
}

// After the stream was synchronised: add the elapsed time of finished stages.
int prof_collect(kmer_analysis* h) {
    if (!profiling(h)) return KMER_OK;
    float* dst[] = {&h->st.ms_scatter, &h->st.ms_repart, &h->st.ms_leaf, &h->st.ms_fallback, &h->st.ms_gate,
                    &h->st.ms_sort};
    uint32_t* cnt[] = {&h->st.n_scatter, &h->st.n_repart, &h->st.n_leaf, &h->st.n_fallback, &h->st.n_gate,
                       &h->st.n_sort};
    for (int i = 0; i < kmer_analysis::STG_N; ++i) {
        if (!h->ev_pending[i]) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev_b[i], h->ev_e[i]));
        *dst[i] += ms;
        *cnt[i] += 1;
        h->ev_pending[i] = false;
    }
    return KMER_OK;
}

// HBM-table recount of the leaves listed by the leaf kernel (leaves of the
// job's bucket window).
int run_fallbacks(kmer_analysis* h, Job& j, unsigned n_fb) {
    if (n_fb == 0) return KMER_OK;
    const unsigned P = j.g.p2 ? job_buckets(j) << j.g.p2 : job_buckets(j);
    std::vector<unsigned> leaves(n_fb);
    CK(cudaMemcpyAsync(leaves.data(), h->fb_list.p, n_fb * 4ull, cudaMemcpyDeviceToHost, h->stream));
    std::vector<unsigned long long> fill(P);
    CK(cudaMemcpyAsync(fill.data(), j.g.p2 ? (const void*)j.l2_fill : (const void*)j.l1_fill, fill.size() * 8,
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    unsigned long long extra_out = 0, max_n = 0;
    for (unsigned e : leaves) {  // a range's records are at most its leaf's
        extra_out += fill[fallback_leaf(e)] / h->p.min_count + 1;
        max_n = std::max(max_n, fill[fallback_leaf(e)]);
    }
    TRY(read_misc(h));
    const unsigned long long out_now = h->host_misc->out_n;
    if (!h->ext_out) TRY(ensure_output(h, out_now + extra_out, out_now));
    fill_job_outputs(h, j);
    const unsigned W = j.g.W;
    const unsigned long long cap = next_pow2(std::max<unsigned long long>(1024, 2 * max_n));
    TRY(h->hbm.ensure(cap * hbm_entry_bytes(W)));
    TRY(prof_begin(h, kmer_analysis::STG_FALLBACK));
    for (unsigned e : leaves) {
        const unsigned long long c = next_pow2(std::max<unsigned long long>(1024, 2 * fill[fallback_leaf(e)]));
        CK(cudaMemsetAsync(h->hbm.p, 0, c * hbm_entry_bytes(W), h->stream));
        CK(launch_records_insert(j, e, h->hbm.p, c, h->num_sms, h->stream));
        CK(launch_hbm_sweep(j, h->hbm.p, c, h->num_sms, h->stream));
        h->st.launches += 2;
    }
    TRY(prof_end(h, kmer_analysis::STG_FALLBACK));
    TRY(read_misc(h));
    TRY(prof_collect(h));
    return status_error(h->host_misc->status);
}

// Totals of the level-2 waves of one pass.
struct WaveTotals {
    unsigned long long out_n = 0, windows = 0, distinct = 0, splits = 0, emitted = 0;
};

// Level-2 stages (repartition, leaves, fallbacks) of one pass over the
// level-1 buckets [b0, b0 + nb) (a wave, or all of them), with their retries.
// `fresh`: reset the device counters first (keeping out_n and the scatter's
// emitted count).  Sets *rescatter when a level-1 bucket overflowed.
int run_level2(kmer_analysis* h, Job j, unsigned b0, unsigned nb, unsigned long long l2_capacity, unsigned cap_max,
               bool fresh, WaveTotals& tot, bool* rescatter) {
    const Geometry g = j.g;
    const unsigned P1 = 1u << g.p1, P2 = 1u << g.p2, W = g.W;
    const unsigned Pw = g.p2 ? nb << g.p2 : nb;  // leaves of the wave
    j.bucket0 = b0;
    j.n_buckets = (b0 == 0 && nb == P1) ? 0 : nb;
    j.l1_start += b0;
    j.l1_cap += b0;
    j.l1_fill += b0;
    std::vector<unsigned long long> exact_leaf;  // exact level-2 layout after an overflow
    if (g.p2) {
        TRY(h->l2_rec.fit(l2_capacity * 8 * W + 64));
        TRY(h->l2_base.ensure(nb * 8ull));
        TRY(h->l2_leafcap.ensure(nb * 4ull));
        TRY(h->l2_fill.ensure(Pw * 8ull));
        TRY(h->tile_prefix.ensure((nb + 1) * 8ull));
        j.l2_rec = h->l2_rec.as<unsigned long long>();
        j.l2_base = h->l2_base.as<unsigned long long>();
        j.l2_leafcap = h->l2_leafcap.as<unsigned int>();
        j.l2_fill = h->l2_fill.as<unsigned long long>();
        j.tile_prefix = h->tile_prefix.as<unsigned long long>();
        j.l2_leaf_start = nullptr;
    }
    TRY(h->split_list.ensure((size_t)Pw * 4));  // every leaf could need key ranges
    fill_job_outputs(h, j);
    if (fresh) TRY(reset_misc(h, tot.out_n, tot.emitted));
    const std::vector<unsigned long long> leaf_off = {0ull, (unsigned long long)Pw};
    TRY(upload(h, h->d_leaf_off, leaf_off));
    TRY(h->d_job_tile_off.ensure(2 * 8));
    for (unsigned sub_attempt = 0;; ++sub_attempt) {
        if (sub_attempt > 8) return fail(KMER_ERR_TABLE_FULL, "leaf buffers still too small after retries");
        j.l2_capacity = exact_leaf.empty() ? l2_capacity : ~0ull;
        TRY(upload(h, h->d_ajob, std::vector<Job>{j}));
        if (g.p2) {
            CK(cudaMemsetAsync(h->l2_fill.p, 0, Pw * 8ull, h->stream));
            TRY(prof_begin(h, kmer_analysis::STG_REPART));
            CK(launch_l2_plan(h->d_ajob.as<Job>(), 1, h->d_job_tile_off.as<unsigned long long>(), h->stream));
            CK(launch_repart(W, h->d_ajob.as<Job>(), h->d_job_tile_off.as<unsigned long long>(), 1, g.p2,
                             h->num_sms, h->stream));
            TRY(prof_end(h, kmer_analysis::STG_REPART));
            h->st.launches += 3;
        }
        TRY(prof_begin(h, kmer_analysis::STG_LEAF));
        CK(launch_leaf(W, h->d_ajob.as<Job>(), h->d_leaf_off.as<unsigned long long>(), 1, Pw, cap_max, h->num_sms,
                       h->stream));
        CK(launch_leaf_split(W, h->d_ajob.as<Job>(), 1, cap_max, h->num_sms, h->stream));
        TRY(prof_end(h, kmer_analysis::STG_LEAF));
        h->st.launches += 2;
        TRY(read_misc(h));
        TRY(prof_collect(h));
        const Misc m = *h->host_misc;
        tot.emitted = m.stats[2];
        if (m.status & ST_L1_OVERFLOW) {  // re-scatter with exact bucket sizes
            *rescatter = true;
            return KMER_OK;
        }
        if (m.status & ST_L2_OVERFLOW) {
            std::vector<unsigned long long> fill(Pw);
            CK(cudaMemcpyAsync(fill.data(), h->l2_fill.p, Pw * 8ull, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            // future queries: more slack, unless only a few leaves overflowed (heavy
            // hitters: the exact layout below takes them; a wider slack for every
            // leaf would only waste memory)
            std::vector<unsigned> leafcap(nb);
            CK(cudaMemcpyAsync(leafcap.data(), h->l2_leafcap.p, nb * 4ull, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            unsigned over = 0;
            for (unsigned i = 0; i < Pw; ++i) over += fill[i] > leafcap[i >> g.p2];
            if (over > std::max(4u, Pw / 64)) h->l2_slack_num = std::min(4096u, h->l2_slack_num * 3 / 2);
            exact_leaf.assign(Pw + 1, 0);
            for (unsigned i = 0; i < Pw; ++i) exact_leaf[i + 1] = exact_leaf[i] + fill[i];
            l2_capacity = exact_leaf[Pw];
            TRY(h->l2_rec.ensure(l2_capacity * 8 * W + 64));
            TRY(h->l2_leaf_start.ensure((Pw + 1) * 8ull));
            CK(cudaMemcpyAsync(h->l2_leaf_start.p, exact_leaf.data(), (Pw + 1) * 8ull, cudaMemcpyHostToDevice,
                               h->stream));
            j.l2_rec = h->l2_rec.as<unsigned long long>();
            j.l2_leaf_start = h->l2_leaf_start.as<unsigned long long>();
            h->st.retries++;
            TRY(reset_misc(h, tot.out_n, m.stats[2]));
            continue;
        }
        if (m.status & (ST_OUT_OVERFLOW | ST_FALLBACK_FULL)) {
            if (m.status & ST_OUT_OVERFLOW) TRY(ensure_output(h, m.out_n + m.out_n / 16 + 1024, tot.out_n));
            if (m.status & ST_FALLBACK_FULL) {
                TRY(h->fb_list.ensure((m.fb_n + 64) * 4ull));
                h->fb_cap = m.fb_n + 64;
            }
            fill_job_outputs(h, j);
            h->st.retries++;
            TRY(reset_misc(h, tot.out_n, m.stats[2]));
            continue;
        }
        TRY(status_error(m.status));
        h->st.fallback_leaves += m.fb_n;
        TRY(run_fallbacks(h, j, m.fb_n));
        const Misc fin = *h->host_misc;
        if (fin.status & ST_OUT_OVERFLOW) return fail(KMER_ERR_CUDA, "fallback output overflow");
        tot.out_n = fin.out_n;
        tot.windows += fin.stats[0];
        tot.distinct += fin.stats[1];
        tot.splits += fin.stats[3];
        return KMER_OK;
    }
}

// One pass of the partitioned variant over every submitted readset: the
// scatter, then the level-2 stages over all level-1 buckets at once, or in
// waves of buckets when their level-2 records do not fit the budget together.
int run_pass(kmer_analysis* h, const Plan& pl, unsigned pass, unsigned cap_max) {
    Geometry g = pl.g;
    const unsigned P1 = 1u << g.p1, P2 = 1u << g.p2;
    const unsigned W = g.W;
    const unsigned long long pass_windows = (pl.windows + pl.passes - 1) / pl.passes;
    std::vector<unsigned long long> caps(P1), starts(P1 + 1);
    const unsigned long long mean = (pass_windows + P1 - 1) / P1;
    {
        // a bucket that still overflows is re-scattered with exact sizes
        const unsigned long long slack = (unsigned long long)(l1_slack(h) * (double)mean) + 1024;
        for (unsigned b = 0; b < P1; ++b) caps[b] = mean + slack;
        // buckets that were far fuller than the rest in the last query of this
        // shape keep their size (scaled to this query's windows)
        if (pl.passes == 1 && h->l1_imb_k == h->p.k && h->l1_prev_p1 == g.p1 && h->l1_prev_fill.size() == P1 &&
            h->l1_prev_windows) {
            const double scale = (double)pass_windows / (double)h->l1_prev_windows;
            for (unsigned b = 0; b < P1; ++b)
                caps[b] = std::max(caps[b], (unsigned long long)(1.02 * scale * (double)h->l1_prev_fill[b]) + 1024);
        }
    }
    const unsigned long long out_start = h->n_out;
    const double slack = (double)h->l2_slack_num / 256.0;
    for (unsigned attempt = 0;; ++attempt) {
        if (attempt > 8) return fail(KMER_ERR_TABLE_FULL, "buffers still too small after %u retries", attempt);
        starts[0] = 0;
        for (unsigned b = 0; b < P1; ++b) starts[b + 1] = starts[b] + caps[b];
        const unsigned long long l1_total = starts[P1];
        if (!h->l1_rec.fits(l1_total * 8 * W + 64)) h->l2_rec.release();  // never both old and new at once
        TRY(h->l1_rec.fit(l1_total * 8 * W + 64));
        // the repartition's bulk copies start on 16-byte boundaries of this region
        if (reinterpret_cast<uintptr_t>(h->l1_rec.p) & 15)
            return fail(KMER_ERR_CUDA, "level-1 record buffer is not 16-byte aligned");
        TRY(h->l1_start.ensure((P1 + 1) * 8));
        TRY(h->l1_cap.ensure(P1 * 8));
        TRY(h->l1_fill.ensure(P1 * 8));
        CK(cudaMemcpyAsync(h->l1_start.p, starts.data(), (P1 + 1) * 8, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->l1_cap.p, caps.data(), P1 * 8, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemsetAsync(h->l1_fill.p, 0, P1 * 8, h->stream));
        // level-2 records of all buckets: sum over buckets of P2 leaves of
        // (mean * slack + 256) records, mean <= n_b / P2 + 1
        const unsigned long long l2_full =
            g.p2 ? (unsigned long long)(slack * (double)(l1_total + (unsigned long long)P1 * P2)) +
                       257ull * P1 * P2 + 1024
                 : 0;
        const size_t l1_bytes = (size_t)l1_total * 8 * W;
        const size_t avail = pl.budget > l1_bytes ? pl.budget - l1_bytes : 0;
        const bool waves = g.p2 && P1 > 1 && (size_t)l2_full * 8 * W > avail;
        if (h->fb_cap < 64) {
            TRY(h->fb_list.ensure(64 * 4));
            h->fb_cap = 64;
        }
        TRY(reset_misc(h, out_start));
        Job j{};
        j.g = g;
        j.pass = pass;
        j.l1_rec = h->l1_rec.as<unsigned long long>();
        j.l1_start = h->l1_start.as<unsigned long long>();
        j.l1_cap = h->l1_cap.as<unsigned long long>();
        j.l1_fill = h->l1_fill.as<unsigned long long>();
        fill_job_outputs(h, j);
        j.l2_slack_num = h->l2_slack_num;
        if (h->p.flags & KMER_FLAG_BLOOM_GATE) {
            j.gate = h->gate2.as<unsigned long long>();
            j.gate_bits = h->gate_bits;
        }
        // one scatter job per submitted readset, one CTA per 256 reads
        std::vector<Job> sjobs;
        std::vector<unsigned long long> tile_off(1, 0);
        for (const kmer_readset* rs : h->submitted) {
            if (rs->n_reads == 0) continue;
            Job js = j;
            set_readset(js, rs);
            sjobs.push_back(js);
            tile_off.push_back(tile_off.back() + (rs->n_reads + 255) / 256);
        }
        TRY(upload(h, h->d_sjobs, sjobs));
        TRY(upload(h, h->d_tile_off, tile_off));
        TRY(prof_begin(h, kmer_analysis::STG_SCATTER));
        if (!sjobs.empty()) {
            CK(launch_scatter(W, h->d_sjobs.as<Job>(), h->d_tile_off.as<unsigned long long>(), (unsigned)sjobs.size(),
                              tile_off.back(), g.p1, g.k, j.gate != nullptr, h->stream));
            h->st.launches++;
        }
        TRY(prof_end(h, kmer_analysis::STG_SCATTER));
        // waves of buckets whose level-2 records fit the budget, from the buckets' fills
        std::vector<unsigned> wave_start = {0, P1};
        unsigned long long l2_cap = l2_full;
        WaveTotals tot;
        tot.out_n = out_start;
        if (waves) {
            TRY(read_misc(h));
            if (h->host_misc->status & ST_L1_OVERFLOW) {
                std::vector<unsigned long long> fill(P1);
                CK(cudaMemcpyAsync(fill.data(), h->l1_fill.p, P1 * 8, cudaMemcpyDeviceToHost, h->stream));
                CK(cudaStreamSynchronize(h->stream));
                for (unsigned b = 0; b < P1; ++b) caps[b] = std::max(caps[b], fill[b]);
                h->st.retries++;
                continue;
            }
            tot.emitted = h->host_misc->stats[2];
            std::vector<unsigned long long> fill(P1);
            CK(cudaMemcpyAsync(fill.data(), h->l1_fill.p, P1 * 8, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            const unsigned long long room = std::max<unsigned long long>(avail / (8ull * W), 1);
            wave_start.assign(1, 0);
            l2_cap = 0;
            unsigned long long cur = 0;
            for (unsigned b = 0; b < P1; ++b) {
                const unsigned long long need =
                    (unsigned long long)(slack * (double)(fill[b] + P2)) + 257ull * P2 + 1024;
                if (b > wave_start.back() && cur + need > room) {
                    wave_start.push_back(b);
                    l2_cap = std::max(l2_cap, cur);
                    cur = 0;
                }
                cur += need;
            }
            l2_cap = std::max(l2_cap, cur);
            wave_start.push_back(P1);
            h->st.l2_waves += (unsigned)wave_start.size() - 1;
        }
        bool rescatter = false;
        for (size_t w = 0; w + 1 < wave_start.size() && !rescatter; ++w)
            TRY(run_level2(h, j, wave_start[w], wave_start[w + 1] - wave_start[w], l2_cap, cap_max, waves, tot,
                           &rescatter));
        if (rescatter) {  // level-1 overflow: take the exact bucket demand and re-scatter
            std::vector<unsigned long long> fill(P1);
            CK(cudaMemcpyAsync(fill.data(), h->l1_fill.p, P1 * 8, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            for (unsigned b = 0; b < P1; ++b) caps[b] = std::max(caps[b], fill[b]);
            h->st.retries++;
            continue;
        }
        if (tot.windows != tot.emitted)  // every emitted window must be counted by exactly one leaf
            return fail(KMER_ERR_CUDA, "internal: %llu windows emitted but %llu counted", tot.emitted, tot.windows);
        if (pass_windows >= (1ull << 26)) {  // learn the buckets' imbalance for the next large query
            std::vector<unsigned long long> fill(P1);
            CK(cudaMemcpyAsync(fill.data(), h->l1_fill.p, P1 * 8, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            const double em = (double)tot.emitted / (double)P1;
            if (em > 0) {
                // the slack of every bucket follows a high quantile (the 99th
                // percentile), not the fullest: a heavy hitter's bucket keeps its
                // own size from l1_prev_fill
                std::vector<unsigned long long> sorted(fill);
                const size_t q = P1 - 1 - P1 / 100;
                std::nth_element(sorted.begin(), sorted.begin() + q, sorted.end());
                h->l1_imbalance = (double)sorted[q] / em;
                h->l1_imb_k = h->p.k;
                h->l1_prev_p1 = g.p1;
                h->l1_prev_fill = pl.passes == 1 ? fill : std::vector<unsigned long long>();
                h->l1_prev_windows = tot.emitted;
            }
        }
        h->n_out = tot.out_n;
        h->res_windows += tot.windows;
        h->res_distinct += tot.distinct;
        h->st.records_emitted += tot.emitted;
        h->st.leaf_splits += tot.splits;
        if (g.p2) h->st.records_l2 += tot.emitted;
        return KMER_OK;
    }
}

// The Bloom gate's pass over every submitted readset (gate.cu): fills F1 and
// F2 and returns the valid windows, first sightings and keys seen at least
// twice.  Filters get 8 bits per expected distinct key (the first sightings
// per window learned at this k, else one per window).
int run_gate(kmer_analysis* h, unsigned long long windows, unsigned long long (&c)[3]) {
    const double ratio = (h->hist_k == h->p.k && h->gate_ratio > 0.0) ? std::min(1.0, 1.15 * h->gate_ratio) : 1.0;
    const unsigned long long keys = std::max<unsigned long long>(1024, (unsigned long long)(ratio * (double)windows));
    unsigned bits = 1;
    while ((1ull << bits) * 64 < keys * 8 && bits < 40) ++bits;
    h->gate_bits = bits;
    const size_t bytes = (size_t)8 << bits;
    TRY(h->gate1.fit(bytes));
    TRY(h->gate2.fit(bytes));
    TRY(h->gate_cnt.ensure(3 * 8));
    CK(cudaMemsetAsync(h->gate1.p, 0, bytes, h->stream));
    CK(cudaMemsetAsync(h->gate2.p, 0, bytes, h->stream));
    CK(cudaMemsetAsync(h->gate_cnt.p, 0, 3 * 8, h->stream));
    Job j{};
    j.g.k = h->p.k;
    j.g.W = h->W();
    j.g.hb = 2 * j.g.k - 64 * (j.g.W - 1);
    TRY(prof_begin(h, kmer_analysis::STG_GATE));
    for (const kmer_readset* rs : h->submitted) {
        if (rs->n_reads == 0) continue;
        set_readset(j, rs);
        CK(launch_gate(j, h->gate1.as<unsigned long long>(), h->gate2.as<unsigned long long>(), bits,
                       h->gate_cnt.as<unsigned long long>(), h->stream));
        h->st.launches++;
    }
    TRY(prof_end(h, kmer_analysis::STG_GATE));
    CK(cudaMemcpyAsync(c, h->gate_cnt.p, sizeof c, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    TRY(prof_collect(h));
    return KMER_OK;
}

int run_direct(kmer_analysis* h, unsigned long long windows) {
    const unsigned W = h->W();
    Geometry g{};
    g.k = h->p.k;
    g.W = W;
    g.hb = 2 * g.k - 64 * (W - 1);
    g.bt = W == 1 ? 2 * g.k : 64;
    const unsigned long long basis = h->p.distinct_hint ? h->p.distinct_hint : windows;
    unsigned long long cap = next_pow2(std::max<unsigned long long>(1024, basis + basis / 3));
    if (!h->ext_out) TRY(ensure_output(h, std::min(windows / h->p.min_count + 1024, basis + 1024), 0));
    for (unsigned attempt = 0;; ++attempt) {
        TRY(h->hbm.ensure(cap * hbm_entry_bytes(W)));
        CK(cudaMemsetAsync(h->hbm.p, 0, cap * hbm_entry_bytes(W), h->stream));
        TRY(reset_misc(h, 0));
        Job j{};
        j.g = g;
        fill_job_outputs(h, j);
        TRY(prof_begin(h, kmer_analysis::STG_SCATTER));
        for (const kmer_readset* rs : h->submitted) {
            if (rs->n_reads == 0) continue;
            set_readset(j, rs);
            CK(launch_direct_insert(j, h->hbm.p, cap, h->stream));
            h->st.launches++;
        }
        TRY(prof_end(h, kmer_analysis::STG_SCATTER));
        TRY(prof_begin(h, kmer_analysis::STG_LEAF));
        CK(launch_hbm_sweep(j, h->hbm.p, cap, h->num_sms, h->stream));
        TRY(prof_end(h, kmer_analysis::STG_LEAF));
        h->st.launches++;
        TRY(read_misc(h));
        TRY(prof_collect(h));
        const Misc m = *h->host_misc;
        if ((m.status & ST_TABLE_FULL) && attempt < 6) {
            cap *= 2;
            h->st.retries++;
            continue;
        }
        if (m.status & ST_OUT_OVERFLOW && attempt < 6) {
            TRY(ensure_output(h, m.out_n + 1024, 0));
            h->st.retries++;
            continue;
        }
        TRY(status_error(m.status));
        h->n_out = m.out_n;
        h->res_windows = m.stats[0];
        h->res_distinct = m.stats[1];
        h->st.records_emitted = m.stats[0];
        return KMER_OK;
    }
}

// Survivors in ascending key order (KMER_FLAG_SORTED_OUTPUT, sort.cu), in
// place in the result arrays.  The scratch is a records or table buffer of the
// query (dead once the survivors are compacted) when one is large enough,
// else a buffer of its own.  Synchronises the stream.
int sort_results(kmer_analysis* h) {
    if (!(h->p.flags & KMER_FLAG_SORTED_OUTPUT) || h->n_out < 2) return KMER_OK;
    if (h->n_out >= 0xFFFFFFFFull) return fail(KMER_ERR_INVALID_ARG, "sorted output limited to 2^32 - 2 survivors");
    const unsigned W = h->W();
    const size_t need = sort_scratch_bytes(W, h->n_out);
    void* scratch = nullptr;
    for (DevBuf* b : {&h->l2_rec, &h->l1_rec, &h->hbm})
        if (!scratch && b->p && b->bytes >= need) scratch = b->p;
    if (!scratch) {
        TRY(h->sort_buf.fit(need));
        scratch = h->sort_buf.p;
    }
    Misc* m = h->misc.as<Misc>();
    CK(cudaMemsetAsync(&m->status, 0, sizeof m->status, h->stream));
    TRY(prof_begin(h, kmer_analysis::STG_SORT));
    unsigned launches = 0;
    CK(launch_sort_survivors(W, h->res_keys, h->res_count, h->res_ext, h->res_cls, h->n_out, h->p.k, scratch,
                             &m->status, h->num_sms, &launches, h->stream));
    TRY(prof_end(h, kmer_analysis::STG_SORT));
    h->st.launches += launches;
    h->lk_cap = 0;  // positions changed
    TRY(read_misc(h));
    TRY(prof_collect(h));
    if (h->host_misc->status & ST_TIMEOUT) return fail(KMER_ERR_TIMEOUT, "the sort's look-back gave up");
    if (h->host_misc->status & ST_SORT_RANGE) return fail(KMER_ERR_CUDA, "internal: sort position out of range");
    return KMER_OK;
}

int do_query(kmer_analysis* h) {
    const auto t0 = std::chrono::steady_clock::now();
    h->have_result = false;
    h->have_contigs = false;
    h->lk_cap = 0;
    h->n_out = h->res_windows = h->res_distinct = 0;
    const kmer_analysis_stats zero{};
    h->st = zero;
    h->st.variant = h->p.variant;
    unsigned long long windows = 0;
    for (const kmer_readset* rs : h->submitted) windows += rs->windows_for(h->p.k);
    if (windows > 0) {
        if (h->p.variant == KMER_VARIANT_HBM_TABLE) {
            TRY(run_direct(h, windows));
            h->st.passes = 1;
        } else {
            const unsigned W = h->W();
            const unsigned cap_max = leaf_table_cap(W, h->leaf_smem_budget);
            size_t budget = h->p.memory_budget;
            if (!budget) budget = (size_t)(0.85 * (double)(free_device_bytes() + h->device_bytes()));
            // output sized from the previous query or a fraction of the windows, at most
            // 35 % of the budget on a first query; grown on demand
            const unsigned long long out_bytes_per = 8ull * W + 4 + 32 + 2;
            const unsigned long long bound = windows / h->p.min_count + 1024;
            unsigned long long want = h->out_hint ? h->out_hint + h->out_hint / 16 + 4096 : windows / 4 + 4096;
            // with min_count 1 every distinct k-mer survives: size for the distinct estimate
            if (!h->out_hint && h->p.min_count == 1)
                want = (h->p.distinct_hint ? std::min<unsigned long long>(h->p.distinct_hint, windows) : windows) + 4096;
            if (!h->out_hint) want = std::min<unsigned long long>(want, 0.35 * (double)budget / out_bytes_per + 4096);
            if (!h->ext_out) TRY(ensure_output(h, std::min(bound, want), 0));
            // the records of a pass get what the output leaves of the budget
            const size_t out_bytes = h->ext_out ? 0 : (size_t)(h->out_cap * out_bytes_per);
            h->hint_ratio = h->p.distinct_hint ? std::min(1.0, (double)h->p.distinct_hint / (double)windows) : 0.0;
            // Bloom gate: the scatter emits only the windows of keys seen twice
            // (windows - first sightings + keys seen twice, up to false positives)
            unsigned long long gate_counts[3] = {0, 0, 0}, rec_windows = windows, gated_distinct = 0;
            size_t rec_budget = budget > 2 * out_bytes ? budget - out_bytes : budget / 2;
            const bool gated = (h->p.flags & KMER_FLAG_BLOOM_GATE) != 0;
            if (gated) {
                TRY(run_gate(h, windows, gate_counts));
                h->st.gate_first = gate_counts[1];
                h->st.gate_twice = gate_counts[2];
                const unsigned long long est = gate_counts[0] - gate_counts[1] + gate_counts[2];
                rec_windows = std::min(windows, est + est / 32 + 4096);
                gated_distinct = gate_counts[2];
                const size_t fb = h->gate1.bytes + h->gate2.bytes;
                rec_budget = rec_budget > 2 * fb ? rec_budget - fb : rec_budget / 2;
            }
            const Plan pl = make_plan(h, rec_windows, rec_budget, cap_max, gated_distinct);
            h->st.pass_bits = pl.g.ps;
            h->st.l1_bits = pl.g.p1;
            h->st.l2_bits = pl.g.p2;
            h->st.leaf_table_slots = cap_max;
            h->st.passes = pl.passes;
            for (unsigned pass = 0; pass < pl.passes; ++pass) TRY(run_pass(h, pl, pass, cap_max));
            if (gated) {  // every valid window was seen by the gate; the leaves saw the gated ones
                h->res_windows = gate_counts[0];
                h->gate_ratio = (double)gate_counts[1] / (double)std::max(1ull, gate_counts[0]);
            }
        }
    }
    TRY(sort_results(h));
    h->out_hint = h->n_out;
    if (h->res_windows) {
        h->hist_k = h->p.k;
        h->hist_ratio = (double)h->res_distinct / (double)h->res_windows;
    }
    h->st.windows = h->res_windows;
    h->st.distinct = h->res_distinct;
    h->st.survivors = h->n_out;
    h->st.device_bytes = h->device_bytes();
    h->st.ms_total = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    h->have_result = true;
    return KMER_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

void kmer::analysis_set_sizing(kmer_analysis_t* h, uint64_t memory_budget, uint64_t distinct_hint) {
    h->p.memory_budget = memory_budget;
    h->p.distinct_hint = distinct_hint;
}

// ====================================================================== C ABI
extern "C" {

void kmer_analysis_default_params(kmer_analysis_params* p, uint32_t k) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->k = k;
    p->min_count = 2;
    p->qual_offset = 33;
    p->qual_threshold = 20;
    p->ext_mode = KMER_EXT_DEPTH_ADAPTIVE;
    p->t_base = 2;
    p->err_num = 1;
    p->err_den = 10;
    p->t_ext = 2;
    p->variant = KMER_VARIANT_PARTITIONED;
}

int kmer_readset_create(const char* bases, const uint8_t* quals, const uint64_t* offsets, uint64_t n_reads,
                        uint32_t qual_offset, uint32_t qual_threshold, int where, void* cuda_stream,
                        kmer_readset_t** out) {
    return make_readset(bases, quals, offsets, n_reads, qual_offset, qual_threshold, where,
                        static_cast<cudaStream_t>(cuda_stream), out);
}

int kmer_readset_pack(kmer_readset_t* rs, const char* bases, const uint8_t* quals, const uint64_t* offsets,
                      uint64_t n_reads, int where, void* cuda_stream) {
    if (!rs) return fail(KMER_ERR_INVALID_ARG, "readset is NULL");
    if (!valid_where(where)) return fail(KMER_ERR_INVALID_ARG, "where must be HOST, DEVICE or HOST_STAGED");
    if (n_reads && (!bases || !quals || !offsets))
        return fail(KMER_ERR_INVALID_ARG, "bases, quals and offsets must be non-NULL when n_reads > 0");
    DeviceGuard dg(rs->device);
    StreamScope scope(static_cast<cudaStream_t>(cuda_stream));
    return pack_readset(rs, bases, quals, offsets, n_reads, where, static_cast<cudaStream_t>(cuda_stream));
}

int kmer_readset_launches(const kmer_readset_t* rs, uint32_t* launches) {
    if (!rs || !launches) return fail(KMER_ERR_INVALID_ARG, "NULL readset or output");
    *launches = rs->launches;
    return KMER_OK;
}

int kmer_readset_info(const kmer_readset_t* rs, uint64_t* n_reads, uint64_t* n_bases) {
    if (!rs) return fail(KMER_ERR_INVALID_ARG, "readset is NULL");
    if (n_reads) *n_reads = rs->n_reads;
    if (n_bases) *n_bases = rs->n_bases;
    return KMER_OK;
}

int kmer_readset_destroy(kmer_readset_t* rs) {
    if (!rs) return KMER_OK;
    DeviceGuard dg(rs->device);
    // analyses on any stream may still read the packed reads
    cudaDeviceSynchronize();
    cudaGetLastError();
    destroy_readset(rs);
    return KMER_OK;
}

int kmer_analysis_create(const kmer_analysis_params* p, void* cuda_stream, kmer_analysis_t** out) {
    if (!out) return fail(KMER_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    TRY(validate_params(p));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(KMER_ERR_NO_DEVICE, "no CUDA device");
    }
    auto* h = new (std::nothrow) kmer_analysis;
    if (!h) return fail(KMER_ERR_OOM, "host allocation failed");
    h->p = *p;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->device = dev;
    int sms = 0, smem_sm = 0, smem_optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(KMER_ERR_NO_DEVICE, "cannot query device %d", dev);
    }
    h->num_sms = sms;
    // two leaf CTAs per SM: half the SM's shared memory minus the per-block reserve and statics
    h->leaf_smem_budget = std::min<size_t>((size_t)smem_optin, (size_t)smem_sm / 2 - 1024 - 256);
    prepare_pool(dev);
    StreamScope scope(h->stream);
    h->host_misc = pinned_misc_get();
    if (!h->host_misc || h->misc.ensure(sizeof(Misc)) != KMER_OK) {
        pinned_misc_put(h->host_misc);
        h->misc.release();
        delete h;
        return fail(KMER_ERR_OOM, "cannot allocate counters");
    }
    *out = h;
    return KMER_OK;
}

int kmer_analysis_submit(kmer_analysis_t* h, const kmer_readset_t* rs) {
    if (!h || !rs) return fail(KMER_ERR_INVALID_ARG, "NULL handle or readset");
    if (rs->qual_offset != h->p.qual_offset || rs->qual_threshold != h->p.qual_threshold)
        return fail(KMER_ERR_INVALID_ARG, "readset packed with qual_offset/threshold %u/%u, analysis uses %u/%u",
                    rs->qual_offset, rs->qual_threshold, h->p.qual_offset, h->p.qual_threshold);
    if (rs->device != h->device) return fail(KMER_ERR_INVALID_ARG, "readset lives on another device");
    h->submitted.push_back(rs);
    h->have_result = false;
    return KMER_OK;
}

int kmer_analysis_submit_raw(kmer_analysis_t* h, const char* bases, const uint8_t* quals, const uint64_t* offsets,
                             uint64_t n_reads, int where) {
    if (!h) return fail(KMER_ERR_INVALID_ARG, "NULL handle");
    DeviceGuard dg(h->device);
    StreamScope scope(h->stream);
    kmer_readset* rs = nullptr;
    TRY(make_readset(bases, quals, offsets, n_reads, h->p.qual_offset, h->p.qual_threshold, where, h->stream, &rs));
    h->owned.push_back(rs);
    h->submitted.push_back(rs);
    h->have_result = false;
    return KMER_OK;
}

int kmer_analysis_query(kmer_analysis_t* h, kmer_result_view* out) {
    if (!h || !out) return fail(KMER_ERR_INVALID_ARG, "NULL handle or output");
    DeviceGuard dg(h->device);
    StreamScope scope(h->stream);
    std::memset(out, 0, sizeof *out);
    int rc = do_query(h);
    if (rc != KMER_OK) {
        h->have_result = false;
        cudaGetLastError();
        return rc;
    }
    out->n = h->n_out;
    out->k = h->p.k;
    out->words = h->W();
    out->keys = reinterpret_cast<const uint64_t*>(h->res_keys);
    out->count = h->res_count;
    out->ext = h->res_ext;
    out->cls = h->res_cls;
    out->windows = h->res_windows;
    out->distinct = h->res_distinct;
    return KMER_OK;
}

int kmer_analysis_query_into(kmer_analysis_t* h, uint64_t* keys, uint32_t* count, uint32_t* ext, uint8_t* cls,
                             uint64_t capacity, int where, kmer_result_view* out) {
    if (!h || !out) return fail(KMER_ERR_INVALID_ARG, "NULL handle or output");
    if (!valid_where(where)) return fail(KMER_ERR_INVALID_ARG, "where must be HOST, DEVICE or HOST_STAGED");
    if (!keys || !count || !ext || !cls) return fail(KMER_ERR_INVALID_ARG, "every output array is required");
    DeviceGuard dg(h->device);
    StreamScope scope(h->stream);
    std::memset(out, 0, sizeof *out);
    // own device buffers, then the copy engines (also for sorted output to
    // page-locked arrays: the sort runs in device memory)
    if (where == KMER_HOST_STAGED || (where == KMER_HOST && (h->p.flags & KMER_FLAG_SORTED_OUTPUT))) {
        const int rc = do_query(h);
        if (rc != KMER_OK) {
            h->have_result = false;
            cudaGetLastError();
            return rc;
        }
        if (h->n_out > capacity)
            return fail(KMER_ERR_INVALID_ARG, "%llu survivors do not fit capacity %llu", h->n_out,
                        (unsigned long long)capacity);
        const unsigned long long n = h->n_out;
        if (n) {
            CK(paced_copy(keys, h->res_keys, n * 8 * h->W(), h->stream));
            CK(paced_copy(count, h->res_count, n * 4, h->stream));
            CK(paced_copy(ext, h->res_ext, n * 32, h->stream));
            CK(paced_copy(cls, h->res_cls, n * 2, h->stream));
        }
        CK(cudaStreamSynchronize(h->stream));
        out->n = n;
        out->k = h->p.k;
        out->words = h->W();
        out->keys = keys;
        out->count = count;
        out->ext = ext;
        out->cls = cls;
        out->windows = h->res_windows;
        out->distinct = h->res_distinct;
        return KMER_OK;
    }
    // the kernels store a survivor's tallies as two 16-byte words and its classes as one 2-byte word
    if ((reinterpret_cast<uintptr_t>(keys) & 7) || (reinterpret_cast<uintptr_t>(count) & 3) ||
        (reinterpret_cast<uintptr_t>(ext) & 15) || (reinterpret_cast<uintptr_t>(cls) & 1))
        return fail(KMER_ERR_INVALID_ARG, "output arrays must be aligned: keys 8, count 4, ext 16, cls 2 bytes");
    void* ptrs[4] = {keys, count, ext, cls};
    if (where == KMER_HOST)
        for (auto& p : ptrs) {
            p = const_cast<void*>(host_mapped(p));
            if (!p) return fail(KMER_ERR_INVALID_ARG, "host output buffers must be page-locked");
        }
    const unsigned long long own_cap = h->out_cap;
    h->ext_out = true;
    h->res_keys = static_cast<unsigned long long*>(ptrs[0]);
    h->res_count = static_cast<unsigned*>(ptrs[1]);
    h->res_ext = static_cast<unsigned*>(ptrs[2]);
    h->res_cls = static_cast<unsigned char*>(ptrs[3]);
    h->out_cap = capacity;
    const int rc = do_query(h);
    h->ext_out = false;
    h->out_cap = own_cap;
    if (rc != KMER_OK) {
        h->have_result = false;
        cudaGetLastError();
        return rc;
    }
    out->n = h->n_out;
    out->k = h->p.k;
    out->words = h->W();
    out->keys = keys;
    out->count = count;
    out->ext = ext;
    out->cls = cls;
    out->windows = h->res_windows;
    out->distinct = h->res_distinct;
    return KMER_OK;
}

int kmer_analysis_copy_results(kmer_analysis_t* h, uint64_t* keys, uint32_t* count, uint32_t* ext, uint8_t* cls,
                               uint64_t capacity) {
    if (!h) return fail(KMER_ERR_INVALID_ARG, "NULL handle");
    if (!h->have_result) return fail(KMER_ERR_BAD_STATE, "no successful query to copy from");
    if (capacity < h->n_out) return fail(KMER_ERR_INVALID_ARG, "capacity %llu < %llu results",
                                         (unsigned long long)capacity, h->n_out);
    DeviceGuard dg(h->device);
    const unsigned long long n = h->n_out;
    if (n) {
        if (keys) CK(paced_copy(keys, h->res_keys, n * 8 * h->W(), h->stream));
        if (count) CK(paced_copy(count, h->res_count, n * 4, h->stream));
        if (ext) CK(paced_copy(ext, h->res_ext, n * 32, h->stream));
        if (cls) CK(paced_copy(cls, h->res_cls, n * 2, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    return KMER_OK;
}

int kmer_analysis_lookup(kmer_analysis_t* h, const uint64_t* keys, uint64_t n, kmer_record* out, int where) {
    if (!h) return fail(KMER_ERR_INVALID_ARG, "NULL handle");
    if (!valid_where(where)) return fail(KMER_ERR_INVALID_ARG, "where must be HOST, DEVICE or HOST_STAGED");
    if (n && (!keys || !out)) return fail(KMER_ERR_INVALID_ARG, "keys and out must be non-NULL when n > 0");
    if (!h->have_result) return fail(KMER_ERR_BAD_STATE, "no successful query to look up in");
    if (h->n_out >= 0xFFFFFFFFull) return fail(KMER_ERR_INVALID_ARG, "index limited to 2^32 - 2 survivors");
    if (n == 0) return KMER_OK;
    DeviceGuard dg(h->device);
    StreamScope scope(h->stream);
    const unsigned W = h->W();
    if (!h->lk_cap) {  // index of the current survivors: a quarter to a half full
        const unsigned long long cap = next_pow2(std::max<unsigned long long>(1024, 2 * h->n_out));
        TRY(h->lk_index.ensure(cap * 4));
        CK(cudaMemsetAsync(h->lk_index.p, 0xFF, cap * 4, h->stream));
        CK(launch_index_build(W, h->res_keys, h->n_out, h->lk_index.as<unsigned>(), cap,
                              h->num_sms, h->stream));
        h->lk_cap = cap;
    }
    const unsigned long long* dq = reinterpret_cast<const unsigned long long*>(keys);
    kmer_record* dout = out;
    if (where == KMER_HOST_STAGED) where = KMER_HOST;  // host arrays are always staged here
    if (where == KMER_HOST) {
        TRY(h->lk_keys.ensure(n * 8 * W));
        TRY(h->lk_out.ensure(n * sizeof(kmer_record)));
        CK(cudaMemcpyAsync(h->lk_keys.p, keys, n * 8 * W, cudaMemcpyHostToDevice, h->stream));
        dq = h->lk_keys.as<unsigned long long>();
        dout = h->lk_out.as<kmer_record>();
    }
    CK(launch_lookup(W, dq, n, h->p.k, h->lk_index.as<unsigned>(), h->lk_cap, h->res_keys, h->res_count, h->res_ext,
                     h->res_cls, dout,
                     h->num_sms, h->stream));
    if (where == KMER_HOST)
        CK(cudaMemcpyAsync(out, dout, n * sizeof(kmer_record), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return KMER_OK;
}

// The survivors' index for lookups, merges and traversals (built once per result).
int ensure_index(kmer_analysis* h) {
    if (h->lk_cap) return KMER_OK;
    const unsigned long long cap = next_pow2(std::max<unsigned long long>(1024, 2 * h->n_out));
    TRY(h->lk_index.ensure(cap * 4));
    CK(cudaMemsetAsync(h->lk_index.p, 0xFF, cap * 4, h->stream));
    CK(launch_index_build(h->W(), h->res_keys, h->n_out, h->lk_index.as<unsigned>(), cap, h->num_sms, h->stream));
    h->lk_cap = cap;
    return KMER_OK;
}

int kmer_analysis_traverse(kmer_analysis_t* h, kmer_contigs_view* out) {
    if (!h || !out) return fail(KMER_ERR_INVALID_ARG, "NULL handle or output");
    if (!h->have_result) return fail(KMER_ERR_BAD_STATE, "no successful query to traverse");
    if (h->n_out > 0x7FFFFFFFull) return fail(KMER_ERR_INVALID_ARG, "traversal limited to 2^31 - 1 k-mers");
    DeviceGuard dg(h->device);
    StreamScope scope(h->stream);
    std::memset(out, 0, sizeof *out);
    const unsigned W = h->W();
    const unsigned long long n = h->n_out;
    TRY(ensure_index(h));
    TRY(h->trav_scratch.fit(traverse_scratch_bytes(n)));
    TRY(h->trav_tot.ensure(16));
    CK(launch_traverse_plan(W, h->res_keys, h->res_cls, n, h->p.k, h->lk_index.as<unsigned>(), h->lk_cap,
                            h->trav_scratch.p, h->trav_tot.as<unsigned long long>(), h->num_sms, h->stream));
    unsigned long long tot[2] = {0, 0};
    CK(cudaMemcpyAsync(tot, h->trav_tot.p, 16, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    TRY(h->trav_bases.fit(tot[0] + 16));
    TRY(h->trav_off.fit((tot[1] + 1) * 8));
    CK(launch_traverse_write(W, h->res_keys, h->res_cls, n, h->p.k, tot[1], h->trav_scratch.p,
                             h->trav_bases.as<char>(), h->trav_off.as<unsigned long long>(), h->num_sms, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->st.launches += 8;
    h->contig_bases = tot[0];
    h->n_contigs = tot[1];
    h->have_contigs = true;
    out->n_contigs = tot[1];
    out->bases = tot[0];
    out->seq = h->trav_bases.as<char>();
    out->offsets = reinterpret_cast<const uint64_t*>(h->trav_off.as<unsigned long long>());
    return KMER_OK;
}

int kmer_analysis_copy_contigs(kmer_analysis_t* h, char* seq, uint64_t* offsets, uint64_t seq_capacity,
                               uint64_t contig_capacity) {
    if (!h) return fail(KMER_ERR_INVALID_ARG, "NULL handle");
    if (!h->have_contigs) return fail(KMER_ERR_BAD_STATE, "no traversal since the last query");
    if (seq_capacity < h->contig_bases || contig_capacity < h->n_contigs)
        return fail(KMER_ERR_INVALID_ARG, "buffers hold %llu bases / %llu contigs, %llu / %llu needed",
                    (unsigned long long)seq_capacity, (unsigned long long)contig_capacity, h->contig_bases,
                    h->n_contigs);
    DeviceGuard dg(h->device);
    StreamScope scope(h->stream);
    if (seq && h->contig_bases) CK(paced_copy(seq, h->trav_bases.p, h->contig_bases, h->stream));
    if (offsets) CK(cudaMemcpyAsync(offsets, h->trav_off.p, (h->n_contigs + 1) * 8, cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return KMER_OK;
}

int kmer_analysis_merge_contigs(kmer_analysis_t* h, const char* contigs, const uint64_t* offsets,
                                uint64_t n_contigs, int where, uint64_t* added, kmer_result_view* out) {
    if (!h || !out) return fail(KMER_ERR_INVALID_ARG, "NULL handle or output");
    if (!valid_where(where)) return fail(KMER_ERR_INVALID_ARG, "where must be HOST, DEVICE or HOST_STAGED");
    if (n_contigs && (!contigs || !offsets)) return fail(KMER_ERR_INVALID_ARG, "NULL contigs with n_contigs > 0");
    if (!h->have_result) return fail(KMER_ERR_BAD_STATE, "no successful query to merge into");
    if (h->res_keys != h->out_keys.as<unsigned long long>())
        return fail(KMER_ERR_BAD_STATE, "the results are in the caller's arrays (query_into): query again first");
    DeviceGuard dg(h->device);
    StreamScope scope(h->stream);
    std::memset(out, 0, sizeof *out);
    if (added) *added = 0;
    const unsigned W = h->W();
    if (n_contigs) {
        if (h->n_out >= 0xFFFFFFFFull) return fail(KMER_ERR_INVALID_ARG, "index limited to 2^32 - 2 survivors");
        // ExtractKmers: the contigs' k-mers as a k-mer analysis of the contigs
        // with every base of high quality (the bases serve as their own quality
        // bytes, offset 0, threshold 0), no count filter, and classes by the
        // static rule with t_ext = 1: a side is UNIQUE when one base follows it
        // anywhere in the contigs, DEAD_END when none, FORK when several
        // A contig longer than kMergePiece bases is cut into pieces of that
        // many bases overlapping by k + 1, since one thread rolls the windows of
        // one read and contigs can be millions of bases long (pieces of 16 k
        // bases, at least 1024: the overlaps cost at most a sixteenth more
        // windows, and the pieces keep the GPU's threads busy).  Each window and
        // both its extension bases then lie whole in some piece; a window at a
        // piece's edge may come twice, once without the base beyond the edge,
        // which adds no base to its sides, and counts are not used.
        const unsigned long long kMergePiece = std::max<unsigned long long>(1024, 16ull * (h->p.k + 1));
        std::vector<unsigned long long> off(n_contigs + 1);
        if (where == KMER_DEVICE) {
            CK(cudaMemcpyAsync(off.data(), offsets, off.size() * 8, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        } else {
            std::memcpy(off.data(), offsets, off.size() * 8);
        }
        std::vector<unsigned long long> psrc, pdst(1, 0);
        bool cut = false;
        for (uint64_t c = 0; c < n_contigs; ++c) {
            const unsigned long long a = off[c], e = off[c + 1];
            if (e < a) return fail(KMER_ERR_INVALID_ARG, "contig offsets decrease at %llu", (unsigned long long)c);
            cut |= e - a > kMergePiece;
            for (unsigned long long st = a;;) {
                const unsigned long long en = std::min(e, st + kMergePiece);
                psrc.push_back(st);
                pdst.push_back(pdst.back() + (en - st));
                if (en >= e) break;
                st = en - (h->p.k + 1);
            }
        }
        DevBuf d_pieces, d_psrc, d_pdst;
        std::vector<char> h_pieces;
        const char* cseq = contigs;
        const uint64_t* coff = offsets;
        uint64_t n_seq = n_contigs;
        int cwhere = where;
        if (cut) {
            const unsigned long long n_p = psrc.size(), bytes = pdst.back();
            if (where == KMER_DEVICE) {
                TRY(d_pieces.ensure(bytes + 16));
                TRY(d_psrc.ensure(n_p * 8));
                TRY(d_pdst.ensure((n_p + 1) * 8));
                CK(cudaMemcpyAsync(d_psrc.p, psrc.data(), n_p * 8, cudaMemcpyHostToDevice, h->stream));
                CK(cudaMemcpyAsync(d_pdst.p, pdst.data(), (n_p + 1) * 8, cudaMemcpyHostToDevice, h->stream));
                CK(launch_piece_copy(contigs, d_psrc.as<unsigned long long>(), d_pdst.as<unsigned long long>(), n_p,
                                     d_pieces.as<char>(), h->num_sms, h->stream));
                h->st.launches++;
                cseq = d_pieces.as<char>();
                coff = reinterpret_cast<const uint64_t*>(d_pdst.p);
            } else {
                h_pieces.resize(bytes);
                for (unsigned long long i = 0; i < n_p; ++i)
                    std::memcpy(h_pieces.data() + pdst[i], contigs + psrc[i], pdst[i + 1] - pdst[i]);
                cseq = h_pieces.data();
                coff = reinterpret_cast<const uint64_t*>(pdst.data());
                cwhere = KMER_HOST_STAGED;
            }
            n_seq = n_p;
        }
        kmer_readset_t* crs = nullptr;
        TRY(make_readset(cseq, reinterpret_cast<const uint8_t*>(cseq), coff, n_seq, 0, 0, cwhere, h->stream, &crs));
        kmer_analysis_params cp;
        kmer_analysis_default_params(&cp, h->p.k);
        cp.min_count = 1;
        cp.qual_offset = 0;
        cp.qual_threshold = 0;
        cp.ext_mode = KMER_EXT_STATIC;
        cp.t_ext = 1;
        kmer_analysis_t* b = nullptr;
        int rc = kmer_analysis_create(&cp, h->stream, &b);
        kmer_result_view bv{};
        if (rc == KMER_OK) rc = kmer_analysis_submit(b, crs);
        if (rc == KMER_OK) rc = kmer_analysis_query(b, &bv);
        if (rc == KMER_OK && !h->lk_cap) {  // index of the current survivors
            const unsigned long long cap = next_pow2(std::max<unsigned long long>(1024, 2 * h->n_out));
            rc = h->lk_index.ensure(cap * 4);
            if (rc == KMER_OK && (cudaMemsetAsync(h->lk_index.p, 0xFF, cap * 4, h->stream) != cudaSuccess ||
                                  launch_index_build(W, h->res_keys, h->n_out, h->lk_index.as<unsigned>(), cap,
                                                     h->num_sms, h->stream) != cudaSuccess))
                rc = fail(KMER_ERR_CUDA, "building the survivors' index failed");
            if (rc == KMER_OK) h->lk_cap = cap;
        }
        const unsigned long long n0 = h->n_out;
        if (rc == KMER_OK) rc = ensure_output(h, n0 + bv.n, n0);
        if (rc == KMER_OK) {
            fill_job_outputs_ptrs(h);
            rc = reset_misc(h, n0);
        }
        if (rc == KMER_OK) {
            Misc* m = h->misc.as<Misc>();
            if (launch_merge_append(W, reinterpret_cast<const unsigned long long*>(bv.keys), bv.cls, bv.n,
                                    h->lk_index.as<unsigned>(), h->lk_cap, h->res_keys, h->res_count, h->res_ext,
                                    h->res_cls, h->out_cap, &m->out_n, &m->status, h->num_sms,
                                    h->stream) != cudaSuccess)
                rc = fail(KMER_ERR_CUDA, "merge kernel launch failed");
            h->st.launches++;
        }
        if (rc == KMER_OK) rc = read_misc(h);
        if (rc == KMER_OK && h->host_misc->status)
            rc = fail(KMER_ERR_CUDA, "internal: merged k-mers past the output capacity");
        if (rc == KMER_OK) {
            h->n_out = h->host_misc->out_n;
            h->lk_cap = 0;  // the index does not cover the added k-mers
            h->have_contigs = false;
            if (added) *added = h->n_out - n0;
            if (h->n_out > n0) rc = sort_results(h);
        }
        if (b) kmer_analysis_destroy(b);
        kmer_readset_destroy(crs);
        if (rc != KMER_OK) {
            h->have_result = false;
            cudaGetLastError();
            return rc;
        }
    }
    out->n = h->n_out;
    out->k = h->p.k;
    out->words = W;
    out->keys = reinterpret_cast<const uint64_t*>(h->res_keys);
    out->count = h->res_count;
    out->ext = h->res_ext;
    out->cls = h->res_cls;
    out->windows = h->res_windows;
    out->distinct = h->res_distinct;
    return KMER_OK;
}

int kmer_analysis_get_stats(const kmer_analysis_t* h, kmer_analysis_stats* out) {
    if (!h || !out) return fail(KMER_ERR_INVALID_ARG, "NULL handle or output");
    *out = h->st;
    return KMER_OK;
}

int kmer_analysis_reset(kmer_analysis_t* h) {
    if (!h) return fail(KMER_ERR_INVALID_ARG, "NULL handle");
    DeviceGuard dg(h->device);
    StreamScope scope(h->stream);
    h->submitted.clear();
    for (kmer_readset* rs : h->owned) destroy_readset(rs);
    h->owned.clear();
    h->have_result = false;
    h->have_contigs = false;
    h->n_out = 0;
    h->lk_cap = 0;
    return KMER_OK;
}

int kmer_analysis_destroy(kmer_analysis_t* h) {
    if (!h) return KMER_OK;
    DeviceGuard dg(h->device);
    StreamScope scope(h->stream);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    kmer_analysis_reset(h);
    DevBuf* bs[] = {&h->l1_rec, &h->l1_start, &h->l1_cap, &h->l1_fill, &h->l2_rec, &h->l2_base, &h->l2_leafcap,
                    &h->l2_fill, &h->l2_leaf_start, &h->tile_prefix, &h->out_keys, &h->out_count, &h->out_ext,
                    &h->out_cls, &h->fb_list, &h->split_list, &h->hbm, &h->misc, &h->lk_index, &h->lk_keys,
                    &h->lk_out};
    for (auto* b : bs) b->release();
    pinned_misc_put(h->host_misc);
    for (int i = 0; i < kmer_analysis::STG_N; ++i) {
        if (h->ev_b[i]) cudaEventDestroy(h->ev_b[i]);
        if (h->ev_e[i]) cudaEventDestroy(h->ev_e[i]);
    }
    delete h;
    return KMER_OK;
}

const char* kmer_strerror(int code) {
    switch (code) {
        case KMER_OK: return "ok";
        case KMER_ERR_INVALID_ARG: return "invalid argument";
        case KMER_ERR_OOM: return "out of memory";
        case KMER_ERR_TABLE_FULL: return "hash table full";
        case KMER_ERR_COUNTER_OVERFLOW: return "counter overflow";
        case KMER_ERR_TIMEOUT: return "device wait timed out";
        case KMER_ERR_CUDA: return "CUDA error";
        case KMER_ERR_BAD_STATE: return "call out of order";
        case KMER_ERR_NO_DEVICE: return "no CUDA device";
    }
    return "unknown error";
}

const char* kmer_last_error_message(void) { return kmer::last_error_message(); }

const char* kmer_version(void) { return "1.0.0"; }

}  // extern "C"
