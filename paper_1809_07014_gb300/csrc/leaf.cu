// Steps a4-a7 fused, one CTA per leaf: the leaf's records are counted in a
// shared-memory open-addressing table (the owner-local histogram of Sec.
// II-A use case 4, with the per-k-mer count and left/right extension tallies
// of Sec. II-B), then the table is swept once: k-mers below min_count are
// dropped, both sides are classified (Sec. II-C) and survivors are compacted
// to the output arrays.
//
// Table slot (SoA): tail word (0 = empty; record tail with the extension
// bits replaced by a mark bit; bit 0 = being published), W-1 head words, a
// 32-bit count and eight 16-bit extension tallies.  A 16-bit tally can only
// wrap if its k-mer's count reaches 65536; the thread that takes a count to
// 65536 flags the leaf, and flagged leaves (and leaves whose distinct keys do
// not fit) are recounted exactly by the HBM-table fallback.
#include "kernels.h"
#include "roll.cuh"

namespace kmer {

constexpr int kLeafThreads = 512;
constexpr unsigned kLeafFull = 1u, kLeafHeavy = 2u, kLeafTimeout = 4u;
constexpr unsigned kSpinLimit = 1u << 22;

__host__ __device__ inline size_t leaf_slot_bytes(unsigned W) { return (size_t)8 * W + 4 + 16; }

size_t leaf_smem_bytes(unsigned W, unsigned cap) { return leaf_slot_bytes(W) * cap + 64; }

unsigned leaf_table_cap(unsigned W, size_t smem_budget) {
    size_t c = (smem_budget - 64) / leaf_slot_bytes(W);
    return (unsigned)(c & ~31ull);
}

template <int W>
__global__ void __launch_bounds__(kLeafThreads, 2) leaf_kernel(const Job j, const unsigned cap_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_claimed, s_flags;
    __shared__ unsigned s_warp[kLeafThreads / 32];
    __shared__ unsigned long long s_base;

    const unsigned leaf = blockIdx.x;
    const Geometry g = j.g;
    unsigned bucket;
    unsigned long long start, n, capr;
    const unsigned long long* recs;
    if (g.p2 == 0) {
        bucket = leaf;
        start = j.l1_start[leaf];
        n = j.l1_fill[leaf];
        capr = j.l1_cap[leaf];
        recs = j.l1_rec;
    } else {
        bucket = leaf >> g.p2;
        const unsigned sub = leaf & ((1u << g.p2) - 1u);
        if (j.l2_leaf_start) {
            start = j.l2_leaf_start[leaf];
            capr = j.l2_leaf_start[leaf + 1] - start;
        } else {
            start = j.l2_base[bucket] + (unsigned long long)sub * j.l2_leafcap[bucket];
            capr = j.l2_leafcap[bucket];
        }
        n = j.l2_fill[leaf];
        recs = j.l2_rec;
    }
    if (n == 0 || n > capr) return;  // an overfull leaf was reported by its writer; the host retries

    unsigned cap = (unsigned)(n + n / 3 + 64 < cap_max ? n + n / 3 + 64 : cap_max);
    unsigned long long* ttail = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* heads = ttail + cap;                     // (W-1) * cap
    unsigned* cnt = reinterpret_cast<unsigned*>(heads + (size_t)(W - 1) * cap);
    unsigned* ext = cnt + cap;                                   // 4 * cap: lanes (A,C),(G,T) left then right
    for (unsigned s = threadIdx.x; s < cap; s += kLeafThreads) ttail[s] = 0ull;
    if (threadIdx.x == 0) { s_claimed = 0; s_flags = 0; }
    __syncthreads();

    const unsigned limit = cap - cap / 8;  // keep probe chains short; fuller leaves go to the fallback
    const unsigned long long* src = recs + start * W;
    for (unsigned long long i = threadIdx.x; i < n; i += kLeafThreads) {
        if (*(volatile unsigned*)&s_flags) break;
        unsigned long long rec[W];
#pragma unroll
        for (int w = 0; w < W; ++w) rec[w] = __ldcs(src + i * W + w);
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
#pragma unroll
                    for (int q = 0; q < 4; ++q) ext[slot * 4 + q] = 0;
#pragma unroll
                    for (int w = 0; w < W - 1; ++w) heads[(size_t)w * cap + slot] = rec[w];
                    __threadfence_block();
                    atomicExch(&ttail[slot], ktail);
                    if (atomicAdd(&s_claimed, 1u) + 1 >= limit) atomicOr(&s_flags, kLeafFull);
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
                    atomicOr(&s_flags, kLeafTimeout);
                    break;
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
            atomicOr(&s_flags, kLeafFull);
            break;
        }
        const unsigned c = atomicAdd(&cnt[found], 1u);
        if (c == 65535u) atomicOr(&s_flags, kLeafHeavy);
        const unsigned l = e5 / 5u, r = e5 - 5u * l;
        if (l) atomicAdd(&ext[found * 4 + ((l - 1) >> 1)], 1u << (16 * ((l - 1) & 1)));
        if (r) atomicAdd(&ext[found * 4 + 2 + ((r - 1) >> 1)], 1u << (16 * ((r - 1) & 1)));
    }
    __syncthreads();
    const unsigned flags = s_flags;
    if (flags & kLeafTimeout) {
        if (threadIdx.x == 0) set_status(j, ST_TIMEOUT);
        return;
    }
    if (flags) {  // table too full or a tally may have wrapped: exact recount in HBM
        if (threadIdx.x == 0) {
            const unsigned idx = atomicAdd(j.fb_n, 1u);
            if (idx < j.fb_cap) j.fb_list[idx] = leaf; else set_status(j, ST_FALLBACK_FULL);
        }
        return;
    }
    if (threadIdx.x == 0) {
        atomicAdd(j.stats + 0, n);
        atomicAdd(j.stats + 1, (unsigned long long)s_claimed);
    }

    // sweep: filter, classify, compact (one global reservation per round)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (unsigned base = 0; base < cap; base += kLeafThreads) {
        const unsigned s = base + threadIdx.x;
        const unsigned long long tl = s < cap ? ttail[s] : 0ull;
        const unsigned c = tl ? cnt[s] : 0u;
        const bool ok = tl != 0ull && c >= j.min_count;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) s_warp[wid] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned run = 0;
            for (int w = 0; w < kLeafThreads / 32; ++w) {
                const unsigned v = s_warp[w];
                s_warp[w] = run;
                run += v;
            }
            s_base = run ? atomicAdd(j.out_n, (unsigned long long)run) : 0ull;
        }
        __syncthreads();
        if (ok) {
            const unsigned long long pos = s_base + s_warp[wid] + __popc(m & ((1u << lane) - 1u));
            if (pos < j.out_cap) {
                unsigned long long key[W];
#pragma unroll
                for (int w = 0; w < W - 1; ++w) key[w] = heads[(size_t)w * cap + s];
                const unsigned long long z = record_z(g, j.pass, bucket, tl);
                key[W - 1] = z_to_tail<W>(z, key, g.bt);
#pragma unroll
                for (int w = 0; w < W; ++w) j.out_keys[pos * W + w] = key[w];
                j.out_count[pos] = c;
                unsigned nl[4], nr[4];
                const unsigned e0 = ext[s * 4 + 0], e1 = ext[s * 4 + 1], e2 = ext[s * 4 + 2], e3 = ext[s * 4 + 3];
                nl[0] = e0 & 0xFFFFu; nl[1] = e0 >> 16; nl[2] = e1 & 0xFFFFu; nl[3] = e1 >> 16;
                nr[0] = e2 & 0xFFFFu; nr[1] = e2 >> 16; nr[2] = e3 & 0xFFFFu; nr[3] = e3 >> 16;
                uint4* eo = reinterpret_cast<uint4*>(j.out_ext + pos * 8);
                eo[0] = make_uint4(nl[0], nl[1], nl[2], nl[3]);
                eo[1] = make_uint4(nr[0], nr[1], nr[2], nr[3]);
                const unsigned char cl = classify_side(nl, c, j), cr = classify_side(nr, c, j);
                reinterpret_cast<uchar2*>(j.out_cls)[pos] = make_uchar2(cl, cr);
            } else {
                set_status(j, ST_OUT_OVERFLOW);
            }
        }
        __syncthreads();
    }
}

template <int W>
static cudaError_t launch_leaf_w(const Job& j, unsigned cap_max, cudaStream_t s) {
    const size_t smem = leaf_smem_bytes(W, cap_max);
    cudaError_t e = cudaFuncSetAttribute(leaf_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned long long leaves = 1ull << (j.g.p1 + j.g.p2);
    leaf_kernel<W><<<(unsigned)leaves, kLeafThreads, smem, s>>>(j, cap_max);
    return cudaGetLastError();
}

cudaError_t launch_leaf(const Job& j, unsigned cap_max, cudaStream_t s) {
    switch (j.g.W) {
        case 1: return launch_leaf_w<1>(j, cap_max, s);
        case 2: return launch_leaf_w<2>(j, cap_max, s);
        case 3: return launch_leaf_w<3>(j, cap_max, s);
        case 4: return launch_leaf_w<4>(j, cap_max, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kmer
