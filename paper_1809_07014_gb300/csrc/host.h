// Host-side internals shared by the C-ABI implementation files (not part of
// the public interface): error reporting, grow-only device buffers, the
// packed readset, small device counters and the planning of one analysis.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "kmer_analysis.h"

namespace kmer {

// Point lookups of n keys against the survivors' index (lookup.cu).
cudaError_t launch_lookup(unsigned W, const unsigned long long* q, unsigned long long n, unsigned k,
                          const unsigned* idx, unsigned long long cap, const unsigned long long* keys,
                          const unsigned* count, const unsigned* ext, const unsigned char* cls, kmer_record* out,
                          int num_sms, cudaStream_t s);

// Records `code` with a formatted detail for kmer_last_error_message().
int fail(int code, const char* fmt, ...);
const char* last_error_message();

#define CK(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return ::kmer::fail(e_ == cudaErrorMemoryAllocation ? KMER_ERR_OOM : KMER_ERR_CUDA,          \
                                "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);    \
    } while (0)

#define TRY(call)                       \
    do {                                \
        int rc_ = (call);               \
        if (rc_ != KMER_OK) return rc_; \
    } while (0)

// Device allocations come from the device's stream-ordered memory pool
// (cudaMallocAsync / cudaFreeAsync), which keeps freed memory for reuse:
// growing or freeing a buffer neither returns memory to the driver nor
// synchronises the device, so analyses on other streams keep running.  The
// stream an allocation is ordered on is the calling thread's current
// allocation stream, set by each API entry point to the stream of the object
// it works on.
extern thread_local cudaStream_t tl_alloc_stream;
struct StreamScope {
    cudaStream_t prev;
    explicit StreamScope(cudaStream_t s) : prev(tl_alloc_stream) { tl_alloc_stream = s; }
    ~StreamScope() { tl_alloc_stream = prev; }
    StreamScope(const StreamScope&) = delete;
    StreamScope& operator=(const StreamScope&) = delete;
};

// Keeps the device's memory pool from trimming itself at synchronisation
// points (once per device).
void prepare_pool(int device);
// Device memory available for new buffers: free memory plus what the pool
// holds unused.
size_t free_device_bytes();

// Grow-only device buffer, allocated on and freed in the order of the stream
// that was current when it was allocated.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; o.bytes = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; s = o.s; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    int ensure(size_t n) {
        if (n <= bytes && p) return KMER_OK;
        release();
        if (n == 0) n = 16;
        s = tl_alloc_stream;
        cudaError_t e = cudaMallocAsync(&p, n, s);
        if (e != cudaSuccess) {
            p = nullptr;
            bytes = 0;
            cudaGetLastError();
            return fail(KMER_ERR_OOM, "allocation of %zu bytes failed: %s", n, cudaGetErrorString(e));
        }
        bytes = n;
        return KMER_OK;
    }
    // Holds n bytes without wasting more than a quarter (plus 64 MB): grows, or
    // shrinks a buffer much larger than needed (device memory held across
    // queries counts against the next query's budget).
    bool fits(size_t n) const { return p && n <= bytes && bytes <= n + n / 4 + (64ull << 20); }
    int fit(size_t n) {
        if (fits(n)) return KMER_OK;
        release();
        return ensure(n);
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

struct Misc {  // small device counters read back after each pass
    unsigned long long out_n;
    unsigned long long stats[4];
    unsigned int status;
    unsigned int fb_n;
    unsigned int split_n;
    unsigned int pad;
};

// Pinned host copies of Misc, from a process-wide pool (allocating and
// freeing pinned memory would synchronise the device).
Misc* pinned_misc_get();
void pinned_misc_put(Misc* m);

inline unsigned long long next_pow2(unsigned long long x) {
    unsigned long long p = 1;
    while (p < x) p <<= 1;
    return p;
}
inline unsigned ceil_log2(unsigned long long x) {
    unsigned b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

// Resizing hints of an existing analysis (its memory budget and expected
// distinct k-mers), for a pooled analysis taken by another request.
void analysis_set_sizing(kmer_analysis_t* h, uint64_t memory_budget, uint64_t distinct_hint);

// Partition geometry for one analysis: k-mer words, pass bits and level bits.
// basis = expected distinct keys (or windows), cap_max = leaf table slots,
// leaf_bits / l1_bits = overrides (0 = automatic).
// Level-2 waves: the repartition and leaf stages may take the level-1 buckets
// in up to this many windows, so that only one window's level-2 records are
// held at a time.
constexpr unsigned kMaxWaves = 8;
Geometry plan_geometry(unsigned k, unsigned long long windows, unsigned long long basis, size_t budget,
                       unsigned cap_max, unsigned leaf_bits, unsigned l1_bits, bool waves, double l1_slack = 0.125);

}  // namespace kmer

struct kmer_readset {
    int device = 0;
    unsigned long long n_reads = 0, n_bases = 0, n_blocks = 0;
    unsigned qual_offset = 33, qual_threshold = 20;
    kmer::DevBuf blocks, blk_off, offsets;
    kmer::DevBuf tmp_bases, tmp_quals, nblk, scratch, stats;  // reused by re-packs
    unsigned launches = 0;
    unsigned long long len_stats[kmer::kLenHist] = {};

    // Exact number of k-windows (before N filtering) for this k.
    unsigned long long windows_for(unsigned k) const {
        unsigned long long w = 0;
        for (unsigned L = k; L < (unsigned)kmer::kLenExact; ++L) w += len_stats[L] * (L - k + 1);
        const unsigned long long big_n = len_stats[kmer::kLenExact], big_sum = len_stats[kmer::kLenExact + 1];
        if (big_n) w += big_sum - (unsigned long long)(k - 1) * big_n;
        return w;
    }
};
