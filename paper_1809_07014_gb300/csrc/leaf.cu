// Steps a4-a7 fused: each leaf (partition) is counted in a shared-memory
// open-addressing table (the owner-local histogram of Sec. II-A use case 4,
// with the per-k-mer count and left/right extension tallies of Sec. II-B),
// then the table is swept once: k-mers below min_count are dropped, both
// sides are classified (Sec. II-C) and survivors are compacted to the output
// arrays.
//
// Persistent CTAs walk the leaves; while one leaf is being swept, the first
// batch of the next leaf's records is already loading into registers.  The
// sweep is per warp: a warp ballots over its slice of the table, lists its
// survivors in shared memory, reserves their output rows with one atomic and
// then writes them with every lane busy (no block barrier in the sweep).
//
// Table slot (SoA, stride = table capacity): tail word (0 = empty; record
// tail with the extension bits replaced by a mark bit; bit 0 = being
// published), W-1 head words, a 32-bit count and eight 16-bit extension
// tallies.  A 16-bit tally can only wrap if its k-mer's count reaches 65536;
// the thread that takes a count to 65536 flags the leaf, and flagged leaves
// (and leaves whose distinct keys do not fit) are recounted exactly by the
// HBM-table fallback.
#include "kernels.h"
#include "roll.cuh"

namespace kmer {

constexpr int kLeafThreads = 512;
constexpr int kLeafWarps = kLeafThreads / 32;
constexpr unsigned kLeafFull = 1u, kLeafHeavy = 2u, kLeafTimeout = 4u;
constexpr unsigned kSpinLimit = 1u << 22;

template <int W>
struct LeafShape {
    static constexpr int U = W <= 2 ? 4 : 2;  // records per thread per batch
    static constexpr int B = U * kLeafThreads;
};

__host__ __device__ inline size_t leaf_slot_bytes(unsigned W) { return (size_t)8 * W + 4 + 16 + 4; }

size_t leaf_smem_bytes(unsigned W, unsigned cap) { return leaf_slot_bytes(W) * cap + 64; }

unsigned leaf_table_cap(unsigned W, size_t smem_budget) {
    size_t c = (smem_budget - 64) / leaf_slot_bytes(W);
    return (unsigned)(c & ~511ull);  // a whole number of warp slices of 32 slots
}

struct LeafInfo {
    unsigned bucket;
    unsigned long long start, n;
    const unsigned long long* recs;
    bool ok;
};

__device__ __forceinline__ LeafInfo leaf_info(const Job& j, unsigned leaf) {
    LeafInfo li;
    unsigned long long capr;
    if (j.g.p2 == 0) {
        li.bucket = leaf;
        li.start = j.l1_start[leaf];
        li.n = j.l1_fill[leaf];
        capr = j.l1_cap[leaf];
        li.recs = j.l1_rec;
    } else {
        li.bucket = leaf >> j.g.p2;
        const unsigned sub = leaf & ((1u << j.g.p2) - 1u);
        if (j.l2_leaf_start) {
            li.start = j.l2_leaf_start[leaf];
            capr = j.l2_leaf_start[leaf + 1] - li.start;
        } else {
            li.start = j.l2_base[li.bucket] + (unsigned long long)sub * j.l2_leafcap[li.bucket];
            capr = j.l2_leafcap[li.bucket];
        }
        li.n = j.l2_fill[leaf];
        li.recs = j.l2_rec;
    }
    // an overfull leaf was reported by its writer and the host retries; skip it
    li.ok = li.n > 0 && li.n <= capr;
    return li;
}

template <int W>
__device__ __forceinline__ void load_batch(const LeafInfo& li, unsigned long long first,
                                           unsigned long long (&r)[LeafShape<W>::U][W]) {
    constexpr int U = LeafShape<W>::U;
    const unsigned long long* src = li.recs + li.start * W;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const unsigned long long i = first + (unsigned long long)u * kLeafThreads + threadIdx.x;
#pragma unroll
        for (int w = 0; w < W; ++w) r[u][w] = (li.ok && i < li.n) ? __ldcs(src + i * W + w) : 0ull;
    }
}

template <int W>
__device__ __forceinline__ void insert_record(const unsigned long long (&rec)[W], unsigned cap, unsigned limit,
                                              unsigned long long* ttail, unsigned long long* heads, unsigned* cnt,
                                              unsigned* ext, unsigned* s_claimed, unsigned* s_flags) {
    const unsigned long long tail = rec[W - 1];
    const unsigned e5 = (unsigned)(tail & 31ull);
    const unsigned long long ktail = (tail & ~63ull) | kKeyMark;
    const unsigned long long zl = tail >> 6;
    unsigned slot = (unsigned)(((unsigned long long)(unsigned)(zl ^ (zl >> 32)) * cap) >> 32);
    int found = -1;
    for (unsigned probe = 0; probe < cap; ++probe) {
        unsigned long long cur = *(volatile unsigned long long*)&ttail[slot];
        if (cur == 0ull) {
            const unsigned long long prev = atomicCAS(&ttail[slot], 0ull, ktail | kBusy);
            if (prev == 0ull) {
                cnt[slot] = 0;
                *reinterpret_cast<uint4*>(&ext[slot * 4]) = make_uint4(0, 0, 0, 0);
#pragma unroll
                for (int w = 0; w < W - 1; ++w) heads[(size_t)w * cap + slot] = rec[w];
                __threadfence_block();
                atomicExch(&ttail[slot], ktail);
                if (atomicAdd(s_claimed, 1u) + 1 >= limit) atomicOr(s_flags, kLeafFull);
                found = (int)slot;
                break;
            }
            cur = prev;
        }
        if ((cur & ~kBusy) == ktail) {
            unsigned spins = 0;
            while (cur & kBusy) {
                if (++spins > kSpinLimit) break;
                cur = *(volatile unsigned long long*)&ttail[slot];
            }
            if (cur & kBusy) {
                atomicOr(s_flags, kLeafTimeout);
                return;
            }
            __threadfence_block();
            bool same = true;
#pragma unroll
            for (int w = 0; w < W - 1; ++w)
                same = same && (*(volatile unsigned long long*)&heads[(size_t)w * cap + slot] == rec[w]);
            if (same) {
                found = (int)slot;
                break;
            }
        }
        slot = slot + 1 == cap ? 0 : slot + 1;
    }
    if (found < 0) {
        atomicOr(s_flags, kLeafFull);
        return;
    }
    const unsigned c = atomicAdd(&cnt[found], 1u);
    if (c == 65535u) atomicOr(s_flags, kLeafHeavy);
    const unsigned l = e5 / 5u, r = e5 - 5u * l;
    if (l) atomicAdd(&ext[found * 4 + ((l - 1) >> 1)], 1u << (16 * ((l - 1) & 1)));
    if (r) atomicAdd(&ext[found * 4 + 2 + ((r - 1) >> 1)], 1u << (16 * ((r - 1) & 1)));
}

template <int W>
__global__ void __launch_bounds__(kLeafThreads, 2) leaf_kernel(const Job j, const unsigned cap_max,
                                                              const unsigned n_leaves) {
    constexpr int U = LeafShape<W>::U, B = LeafShape<W>::B;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_claimed, s_flags;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    unsigned leaf = blockIdx.x;
    if (leaf >= n_leaves) return;
    LeafInfo li = leaf_info(j, leaf);
    unsigned long long batch[U][W];
    load_batch<W>(li, 0, batch);

    for (;;) {
        // ---------------------------------------------------------- count
        if (li.ok) {
            const unsigned long long n = li.n;
            const unsigned long long want = ((n * j.table_ratio_num) >> 16) + 512;
            const unsigned cap = (unsigned)(want < cap_max ? ((want + 511) & ~511ull) : cap_max);
            unsigned long long* ttail = reinterpret_cast<unsigned long long*>(smem);
            unsigned long long* heads = ttail + cap;
            unsigned* cnt = reinterpret_cast<unsigned*>(heads + (size_t)(W - 1) * cap);
            unsigned* ext = cnt + cap;
            unsigned* list = ext + 4 * (size_t)cap;
            for (unsigned s = threadIdx.x; s < cap; s += kLeafThreads) ttail[s] = 0ull;
            if (threadIdx.x == 0) { s_claimed = 0; s_flags = 0; }
            __syncthreads();
            const unsigned limit = cap - cap / 8;  // keep probe chains short; fuller leaves go to the fallback
            for (unsigned long long first = 0; first < n; first += B) {
                if (first) load_batch<W>(li, first, batch);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const unsigned long long i = first + (unsigned long long)u * kLeafThreads + threadIdx.x;
                    if (i < n && !*(volatile unsigned*)&s_flags)
                        insert_record<W>(batch[u], cap, limit, ttail, heads, cnt, ext, &s_claimed, &s_flags);
                }
            }
            __syncthreads();
            const unsigned flags = s_flags;
            const unsigned claimed = s_claimed;
            // the next leaf's first batch loads while this one is swept
            const unsigned next = leaf + gridDim.x;
            LeafInfo nli;
            nli.ok = false;
            if (next < n_leaves) {
                nli = leaf_info(j, next);
                load_batch<W>(nli, 0, batch);
            }
            if (flags & kLeafTimeout) {
                if (threadIdx.x == 0) set_status(j, ST_TIMEOUT);
            } else if (flags) {  // table too full or a tally may have wrapped: exact recount in HBM
                if (threadIdx.x == 0) {
                    const unsigned idx = atomicAdd(j.fb_n, 1u);
                    if (idx < j.fb_cap) j.fb_list[idx] = leaf; else set_status(j, ST_FALLBACK_FULL);
                }
            } else {
                if (threadIdx.x == 0) {
                    atomicAdd(j.stats + 0, n);
                    atomicAdd(j.stats + 1, (unsigned long long)claimed);
                }
                // ------------------------------------------------------ sweep (per warp)
                const unsigned per = cap / kLeafWarps;  // a multiple of 32
                const unsigned s0 = wid * per;
                unsigned* mylist = list + s0;
                unsigned count = 0;
                for (unsigned s = s0 + lane; s < s0 + per; s += 32) {
                    const unsigned long long tl = ttail[s];
                    const bool ok = tl != 0ull && cnt[s] >= j.min_count;
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    if (ok) mylist[count + __popc(m & ((1u << lane) - 1u))] = s;
                    count += __popc(m);
                }
                __syncwarp();
                unsigned long long wbase = 0;
                if (lane == 0 && count) wbase = atomicAdd(j.out_n, (unsigned long long)count);
                wbase = __shfl_sync(0xffffffffu, wbase, 0);
                for (unsigned i = lane; i < count; i += 32) {
                    const unsigned s = mylist[i];
                    const unsigned long long pos = wbase + i;
                    if (pos >= j.out_cap) {
                        set_status(j, ST_OUT_OVERFLOW);
                        continue;
                    }
                    const unsigned long long tl = ttail[s];
                    const unsigned c = cnt[s];
                    unsigned long long key[W];
#pragma unroll
                    for (int w = 0; w < W - 1; ++w) key[w] = heads[(size_t)w * cap + s];
                    const unsigned long long z = record_z(j.g, j.pass, li.bucket, tl);
                    key[W - 1] = z_to_tail<W>(z, key, j.g.bt);
#pragma unroll
                    for (int w = 0; w < W; ++w) j.out_keys[pos * W + w] = key[w];
                    j.out_count[pos] = c;
                    const uint4 e = *reinterpret_cast<const uint4*>(&ext[s * 4]);
                    unsigned nl[4] = {e.x & 0xFFFFu, e.x >> 16, e.y & 0xFFFFu, e.y >> 16};
                    unsigned nr[4] = {e.z & 0xFFFFu, e.z >> 16, e.w & 0xFFFFu, e.w >> 16};
                    uint4* eo = reinterpret_cast<uint4*>(j.out_ext + pos * 8);
                    eo[0] = make_uint4(nl[0], nl[1], nl[2], nl[3]);
                    eo[1] = make_uint4(nr[0], nr[1], nr[2], nr[3]);
                    reinterpret_cast<uchar2*>(j.out_cls)[pos] =
                        make_uchar2(classify_side(nl, c, j), classify_side(nr, c, j));
                }
            }
            __syncthreads();  // the table is reused by the next leaf
            leaf = next;
            li = nli;
        } else {
            const unsigned next = leaf + gridDim.x;
            if (next >= n_leaves) break;
            leaf = next;
            li = leaf_info(j, leaf);
            load_batch<W>(li, 0, batch);
            continue;
        }
        if (leaf >= n_leaves) break;
    }
}

template <int W>
static cudaError_t launch_leaf_w(const Job& j, unsigned cap_max, int num_sms, cudaStream_t s) {
    const size_t smem = leaf_smem_bytes(W, cap_max);
    cudaError_t e = cudaFuncSetAttribute(leaf_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned long long leaves = 1ull << (j.g.p1 + j.g.p2);
    unsigned long long grid = (unsigned long long)num_sms * 2;
    if (grid > leaves) grid = leaves;
    leaf_kernel<W><<<(unsigned)grid, kLeafThreads, smem, s>>>(j, cap_max, (unsigned)leaves);
    return cudaGetLastError();
}

cudaError_t launch_leaf(const Job& j, unsigned cap_max, int num_sms, cudaStream_t s) {
    switch (j.g.W) {
        case 1: return launch_leaf_w<1>(j, cap_max, num_sms, s);
        case 2: return launch_leaf_w<2>(j, cap_max, num_sms, s);
        case 3: return launch_leaf_w<3>(j, cap_max, num_sms, s);
        case 4: return launch_leaf_w<4>(j, cap_max, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kmer
