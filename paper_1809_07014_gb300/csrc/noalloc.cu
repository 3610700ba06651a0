// k-mer analysis for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a memory
// pool or allocator hook that must not recurse into the allocator, plugins
// whose host application owns every device allocation, or latency-critical
// paths where an allocation (and the device synchronisation it may imply) is
// not allowed.  For them this file offers one entry point whose only device
// scratch is a file-scope static array, reserved once when the library is
// loaded on a device and held until the process exits.
//
// The computation is the HBM-table variant of k-mer analysis (every window
// inserted into one open-addressing table, then the table swept), reading
// the ASCII bases and qualities directly, so that no packed copy is needed.
// The table lives in the static array, which bounds the input size.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kmer_analysis.h"

namespace kmer {
namespace {

// 32 MiB of device scratch: a 256-byte header of counters, then the table.
constexpr size_t kNoAllocScratchBytes = 32ull << 20;
constexpr size_t kNoAllocHeader = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NaCounters {
    unsigned long long out_n;
    unsigned int status;
};

// A read whose offsets decrease or leave [offsets[0], offsets[n_reads]]:
// skipped without touching its bases, and the call returns INVALID_ARG.
constexpr unsigned kNaBadOffsets = 1u << 8;

constexpr unsigned long long kNaOcc = 1ull << 63, kNaPub = 1ull << 62;
constexpr unsigned kNaSpinLimit = 1u << 22;

template <int W>
struct __align__(8) NaEntry {
    unsigned long long key[W];
    unsigned count;
    unsigned pad;
    unsigned ext[8];
};

__host__ __device__ inline size_t na_entry_bytes(unsigned W) { return 8ull * W + 40; }

// Largest power-of-two slot count whose table fits after the header.
__host__ __device__ inline unsigned long long na_slots(unsigned W) {
    unsigned long long c = 1;
    while ((c * 2) * na_entry_bytes(W) <= kNoAllocScratchBytes - kNoAllocHeader) c *= 2;
    return c;
}
// Largest input accepted: every window distinct still fills at most 3/4 of the table.
__host__ __device__ inline unsigned long long na_max_bases(unsigned W) { return na_slots(W) / 4 * 3; }

template <int W>
__device__ bool na_insert(NaEntry<W>* t, unsigned long long cap, const unsigned long long (&key)[W],
                          unsigned long long z, unsigned lcode, unsigned rcode, NaCounters* c) {
    // home slot from the top bits of a multiplicative hash of z (the low bits
    // of a one-word z depend only on the low bits of the key)
    unsigned long long slot = (z * 0x9E3779B97F4A7C15ull) >> (__clzll(cap) + 1);
    const unsigned long long k0 = key[0] | kNaOcc;
    for (unsigned long long probe = 0; probe < cap; ++probe) {
        NaEntry<W>* e = t + slot;
        unsigned long long cur = *(volatile unsigned long long*)&e->key[0];
        bool hit = false;
        if (cur == 0ull) {
            const unsigned long long prev = atomicCAS(&e->key[0], 0ull, W == 1 ? k0 : (k0 | kNaPub));
            if (prev == 0ull) {
                if (W > 1) {
#pragma unroll
                    for (int w = 1; w < W; ++w) e->key[w] = key[w];
                    __threadfence();
                    atomicExch(&e->key[0], k0);
                }
                hit = true;
            } else {
                cur = prev;
            }
        }
        if (!hit && (cur & ~kNaPub) == k0) {
            hit = true;
            if (W > 1) {
                unsigned spins = 0;
                while (cur & kNaPub) {
                    if (++spins > kNaSpinLimit) {
                        atomicOr(&c->status, ST_TIMEOUT);
                        return false;
                    }
                    cur = *(volatile unsigned long long*)&e->key[0];
                }
                __threadfence();
#pragma unroll
                for (int w = 1; w < W; ++w) hit = hit && (*(volatile unsigned long long*)&e->key[w] == key[w]);
            }
        }
        if (hit) {
            const unsigned old = atomicAdd(&e->count, 1u);
            if (old == 0xFFFFFFFFu) atomicOr(&c->status, ST_COUNTER_OVERFLOW);
            if (lcode) atomicAdd(&e->ext[lcode - 1], 1u);
            if (rcode) atomicAdd(&e->ext[3 + rcode], 1u);
            return true;
        }
        slot = (slot + 1) & (cap - 1);
    }
    atomicOr(&c->status, ST_TABLE_FULL);
    return false;
}

// One thread per read: roll the forward k-mer and its reverse complement over
// the ASCII bases and insert every window without N (same window, canonical
// and extension rules as the packed path).
template <int W>
__global__ void __launch_bounds__(256) noalloc_insert_kernel(const char* __restrict__ bases,
                                                            const unsigned char* __restrict__ quals,
                                                            const unsigned long long* __restrict__ offsets,
                                                            unsigned long long n_reads, unsigned long long span0,
                                                            unsigned long long span1, unsigned k,
                                                            unsigned qual_offset, unsigned qual_threshold,
                                                            unsigned char* scratch) {
    NaCounters* cnt = reinterpret_cast<NaCounters*>(scratch);
    NaEntry<W>* table = reinterpret_cast<NaEntry<W>*>(scratch + kNoAllocHeader);
    const unsigned long long cap = na_slots(W);
    const unsigned hb = 2 * k - 64 * (W - 1);
    const unsigned bt = W == 1 ? 2 * k : 64;
    const unsigned long long topmask = low_mask(hb);
    const unsigned long long r = blockIdx.x * 256ull + threadIdx.x;
    if (r < n_reads) {
        const unsigned long long a = offsets[r], e = offsets[r + 1];
        // only the span [offsets[0], offsets[n_reads]) was checked by the host
        if (a < span0 || e < a || e > span1) {
            atomicOr(&cnt->status, kNaBadOffsets);
            return;
        }
        const unsigned long long L = e - a;
        unsigned long long fwd[W], rc[W];
#pragma unroll
        for (int w = 0; w < W; ++w) { fwd[w] = 0; rc[w] = 0; }
        unsigned long long gh0 = 0, gh1 = 0;
        long long last_n = -1;
        unsigned out = 0;
        for (unsigned long long t = 0; t <= L; ++t) {
            unsigned b = 0, good = 0, isn = 0;
            if (t < L) {
                const unsigned char ch = (unsigned char)bases[a + t];
                const unsigned q = quals[a + t];
                switch (ch) {
                    case 'A': b = 0; break;
                    case 'C': b = 1; break;
                    case 'G': b = 2; break;
                    case 'T': b = 3; break;
                    default: isn = 1; break;
                }
                good = (!isn && q >= qual_offset && q - qual_offset >= qual_threshold) ? 1u : 0u;
            }
            if (t >= k && last_n < (long long)(t - k)) {
                const unsigned long long i = t - k;
                const unsigned lgood = k < 64 ? (unsigned)(gh0 >> k) & 1u : (unsigned)(gh1 >> (k - 64)) & 1u;
                unsigned lc = (i >= 1 && lgood) ? out + 1 : 0;
                unsigned rcd = (t < L && good) ? b + 1 : 0;
                bool flip = false;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    if (fwd[w] != rc[w]) { flip = rc[w] < fwd[w]; break; }
                }
                unsigned long long key[W];
#pragma unroll
                for (int w = 0; w < W; ++w) key[w] = flip ? rc[w] : fwd[w];
                if (flip) {
                    const unsigned nl = rcd ? 5 - rcd : 0, nr = lc ? 5 - lc : 0;
                    lc = nl;
                    rcd = nr;
                }
                const unsigned long long z = key_to_z<W>(key, bt);
                if (!na_insert<W>(table, cap, key, z, lc, rcd, cnt)) break;
            }
            if (t < L) {
                out = (unsigned)(fwd[0] >> (hb - 2)) & 3u;
#pragma unroll
                for (int w = 0; w < W - 1; ++w) fwd[w] = (fwd[w] << 2) | (fwd[w + 1] >> 62);
                fwd[W - 1] = (fwd[W - 1] << 2) | b;
                fwd[0] &= topmask;
#pragma unroll
                for (int w = W - 1; w > 0; --w) rc[w] = (rc[w] >> 2) | (rc[w - 1] << 62);
                rc[0] = (rc[0] >> 2) | ((unsigned long long)(3u - b) << (hb - 2));
                gh1 = (gh1 << 1) | (gh0 >> 63);
                gh0 = (gh0 << 1) | good;
                if (isn) last_n = (long long)t;
            }
        }
    }
}

template <int W>
__global__ void __launch_bounds__(256) noalloc_sweep_kernel(unsigned char* scratch, unsigned min_count,
                                                           Job cls_params, unsigned long long* keys,
                                                           unsigned* count, unsigned* ext, unsigned char* cls,
                                                           unsigned long long capacity) {
    NaCounters* cnt = reinterpret_cast<NaCounters*>(scratch);
    const NaEntry<W>* table = reinterpret_cast<const NaEntry<W>*>(scratch + kNoAllocHeader);
    const unsigned long long cap = na_slots(W);
    const int lane = threadIdx.x & 31;
    for (unsigned long long base = blockIdx.x * 256ull + (threadIdx.x & ~31u); base < cap;
         base += (unsigned long long)gridDim.x * 256) {
        const unsigned long long s = base + lane;
        const NaEntry<W>* e = table + s;
        const unsigned long long k0 = s < cap ? e->key[0] : 0ull;
        const unsigned c = k0 ? e->count : 0u;
        const bool ok = k0 != 0ull && c >= min_count;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        unsigned long long wbase = 0;
        if (lane == 0 && m) wbase = atomicAdd(&cnt->out_n, (unsigned long long)__popc(m));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (ok) {
            const unsigned long long pos = wbase + __popc(m & ((1u << lane) - 1u));
            if (pos < capacity) {
                keys[pos * W] = k0 & ~(kNaOcc | kNaPub);
#pragma unroll
                for (int w = 1; w < W; ++w) keys[pos * W + w] = e->key[w];
                count[pos] = c;
                unsigned nl[4], nr[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) { nl[b] = e->ext[b]; nr[b] = e->ext[4 + b]; }
#pragma unroll
                for (int b = 0; b < 4; ++b) { ext[pos * 8 + b] = nl[b]; ext[pos * 8 + 4 + b] = nr[b]; }
                cls[pos * 2] = classify_side(nl, c, cls_params);
                cls[pos * 2 + 1] = classify_side(nr, c, cls_params);
            }
        }
    }
}

// Device address of the static array, looked up once per device and CUDA
// context: a module's symbol address belongs to the context that loaded it,
// so a caller that runs this function under a context of its own, or after
// cudaDeviceReset, gets the address in the context current at the call.
struct ScratchAddr {
    int dev;
    CUcontext ctx;
    unsigned char* ptr;
};
std::vector<ScratchAddr> g_scratch_addrs;
std::mutex g_scratch_mu;
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;

int scratch_for_device(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_ctx_get_current) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return KMER_ERR_CUDA;
        }
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return KMER_ERR_NO_DEVICE;
    for (const ScratchAddr& a : g_scratch_addrs)
        if (a.dev == dev && a.ctx == ctx) {
            *out = a.ptr;
            return KMER_OK;
        }
    void* p = nullptr;
    // the host-side name of the array is only a stand-in: ask the runtime for its device address
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return KMER_ERR_CUDA;
    }
    g_scratch_addrs.push_back({dev, ctx, static_cast<unsigned char*>(p)});
    *out = static_cast<unsigned char*>(p);
    return KMER_OK;
}

template <int W>
cudaError_t launch_noalloc(const char* bases, const uint8_t* quals, const uint64_t* offsets, uint64_t n_reads,
                           const unsigned long long (&span)[2], const kmer_analysis_params* p,
                           unsigned char* scratch, uint64_t* keys, uint32_t* count, uint32_t* ext, uint8_t* cls,
                           uint64_t capacity, cudaStream_t s) {
    if (n_reads) {
        noalloc_insert_kernel<W><<<(unsigned)((n_reads + 255) / 256), 256, 0, s>>>(
            bases, quals, reinterpret_cast<const unsigned long long*>(offsets), n_reads, span[0], span[1], p->k,
            p->qual_offset, p->qual_threshold, scratch);
    }
    Job cp{};
    cp.ext_mode = p->ext_mode;
    cp.t_base = p->t_base;
    cp.err_num = p->err_num;
    cp.err_den = p->err_den;
    cp.t_ext = p->t_ext;
    const unsigned long long grid = (na_slots(W) + 255) / 256;
    noalloc_sweep_kernel<W><<<(unsigned)(grid < 1184 ? grid : 1184), 256, 0, s>>>(
        scratch, p->min_count, cp, reinterpret_cast<unsigned long long*>(keys), count, ext, cls, capacity);
    return cudaGetLastError();
}

}  // namespace
}  // namespace kmer

using namespace kmer;

extern "C" int kmer_analysis_run_noalloc(const char* bases, const uint8_t* quals, const uint64_t* offsets,
                                         uint64_t n_reads, const kmer_analysis_params* p, uint64_t* keys,
                                         uint32_t* count, uint32_t* ext, uint8_t* cls, uint64_t capacity,
                                         uint64_t* n_out, void* cuda_stream) {
    if (!p || !n_out) return KMER_ERR_INVALID_ARG;
    *n_out = 0;
    if (p->k == 0 || p->k > KMER_MAX_K || p->k % 2 == 0 || p->min_count == 0 || p->ext_mode > 1 ||
        (p->ext_mode == 0 && p->err_den == 0) || p->qual_offset > 255 || p->qual_threshold > 255)
        return KMER_ERR_INVALID_ARG;
    if (n_reads && (!bases || !quals || !offsets)) return KMER_ERR_INVALID_ARG;
    if (capacity && (!keys || !count || !ext || !cls)) return KMER_ERR_INVALID_ARG;
    const unsigned W = (2 * p->k + 63) / 64;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return KMER_ERR_NO_DEVICE;
    }
    unsigned char* scratch = nullptr;
    int rc = scratch_for_device(dev, &scratch);
    if (rc != KMER_OK) return rc;
    // input size: bases spanned by the reads, read from the device (8 bytes each, no allocation)
    unsigned long long span[2] = {0, 0};
    if (n_reads) {
        if (cudaMemcpyAsync(&span[0], offsets, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&span[1], offsets + n_reads, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return KMER_ERR_CUDA;
        }
        if (span[1] < span[0]) return KMER_ERR_INVALID_ARG;
        if (span[1] - span[0] > na_max_bases(W)) return KMER_ERR_INVALID_ARG;  // beyond the static table
    }
    // the table and counters must start at zero; earlier calls left their contents behind
    const size_t used = kNoAllocHeader + na_slots(W) * na_entry_bytes(W);
    if (cudaMemsetAsync(scratch, 0, used, s) != cudaSuccess) {
        cudaGetLastError();
        return KMER_ERR_CUDA;
    }
    cudaError_t e;
    switch (W) {
        case 1: e = launch_noalloc<1>(bases, quals, offsets, n_reads, span, p, scratch, keys, count, ext, cls, capacity, s); break;
        case 2: e = launch_noalloc<2>(bases, quals, offsets, n_reads, span, p, scratch, keys, count, ext, cls, capacity, s); break;
        case 3: e = launch_noalloc<3>(bases, quals, offsets, n_reads, span, p, scratch, keys, count, ext, cls, capacity, s); break;
        default: e = launch_noalloc<4>(bases, quals, offsets, n_reads, span, p, scratch, keys, count, ext, cls, capacity, s); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KMER_ERR_CUDA;
    }
    NaCounters c{};
    if (cudaMemcpyAsync(&c, scratch, sizeof c, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return KMER_ERR_CUDA;
    }
    if (c.status & kNaBadOffsets) return KMER_ERR_INVALID_ARG;  // nothing of the call is usable
    *n_out = c.out_n;
    if (c.status & ST_TIMEOUT) return KMER_ERR_TIMEOUT;
    if (c.status & ST_COUNTER_OVERFLOW) return KMER_ERR_COUNTER_OVERFLOW;
    if (c.status & ST_TABLE_FULL) return KMER_ERR_TABLE_FULL;
    if (c.out_n > capacity) return KMER_ERR_INVALID_ARG;  // *n_out tells the caller how much room is needed
    return KMER_OK;
}

