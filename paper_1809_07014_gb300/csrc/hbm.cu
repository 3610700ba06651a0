// Open-addressing hash table in HBM with 32-bit counters: the global
// counting histogram of Sec. II-B on one GPU.  It serves two purposes: the
// "direct" variant (every window of the reads inserted straight into one
// table), and the exact fallback for leaves whose distinct k-mers did not fit
// a shared-memory table or whose 16-bit tallies could wrap.
//
// Entry: W key words (canonical key, word 0 tagged with bit 63 = occupied,
// bit 62 = being published; both are free because word 0 holds at most 62
// key bits for odd k), a 32-bit count, eight 32-bit tallies.  The table is
// zeroed before use.  Claiming a slot is one 64-bit CAS on word 0; for W > 1
// the other words are written before word 0 is published, and a reader that
// meets a slot being published waits a bounded number of polls.
#include "kernels.h"
#include "roll.cuh"

namespace kmer {

constexpr unsigned long long kOcc = 1ull << 63, kPub = 1ull << 62;
constexpr unsigned kHbmSpinLimit = 1u << 22;

template <int W>
struct __align__(8) HEntry {
    unsigned long long key[W];
    unsigned count;
    unsigned pad;
    unsigned ext[8];
};

size_t hbm_entry_bytes(unsigned W) {
    switch (W) {
        case 1: return sizeof(HEntry<1>);
        case 2: return sizeof(HEntry<2>);
        case 3: return sizeof(HEntry<3>);
        default: return sizeof(HEntry<4>);
    }
}

// Adds `mult` windows of one key with the same extension codes.
template <int W>
__device__ bool hbm_insert(HEntry<W>* t, unsigned long long cap, const unsigned long long (&key)[W],
                           unsigned long long z, unsigned lcode, unsigned rcode, unsigned* status,
                           unsigned mult = 1) {
    // home slot from the top bits of a multiplicative hash of z (the low bits
    // of a one-word z depend only on the low bits of the key)
    unsigned long long slot = (z * 0x9E3779B97F4A7C15ull) >> (__clzll(cap) + 1);
    const unsigned long long k0 = key[0] | kOcc;
    for (unsigned long long probe = 0; probe < cap; ++probe) {
        HEntry<W>* e = t + slot;
        unsigned long long cur = *(volatile unsigned long long*)&e->key[0];
        bool hit = false;
        if (cur == 0ull) {
            const unsigned long long prev = atomicCAS(&e->key[0], 0ull, W == 1 ? k0 : (k0 | kPub));
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
        if (!hit && (cur & ~kPub) == k0) {
            hit = true;
            if (W > 1) {
                unsigned spins = 0;
                while (cur & kPub) {
                    if (++spins > kHbmSpinLimit) {
                        atomicOr(status, ST_TIMEOUT);
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
            const unsigned old = atomicAdd(&e->count, mult);
            if (old > 0xFFFFFFFFu - mult) atomicOr(status, ST_COUNTER_OVERFLOW);
            if (lcode) atomicAdd(&e->ext[lcode - 1], mult);
            if (rcode) atomicAdd(&e->ext[3 + rcode], mult);
            return true;
        }
        slot = (slot + 1) & (cap - 1);
    }
    atomicOr(status, ST_TABLE_FULL);
    return false;
}

// Direct variant: one thread per read, every window inserted into the table.
template <int W>
__global__ void __launch_bounds__(256) direct_insert_kernel(const Job j, HEntry<W>* t, unsigned long long cap) {
    const unsigned long long r = blockIdx.x * 256ull + threadIdx.x;
    unsigned windows = 0;
    if (r < j.n_reads) {
        Roll<W> roll;
        roll.init(j, r);
        for (unsigned long long step = 0; step <= roll.L; ++step) {
            unsigned long long key[W];
            unsigned lc, rc;
            if (roll.step(step, key, lc, rc)) {
                const unsigned long long z = key_to_z<W>(key, j.g.bt);
                if (!hbm_insert<W>(t, cap, key, z, lc, rc, j.status)) break;
                ++windows;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) windows += __shfl_xor_sync(0xffffffffu, windows, o);
    if ((threadIdx.x & 31) == 0 && windows) atomicAdd(j.stats + 0, (unsigned long long)windows);
}

// Fallback: the records of one key range of a leaf (fallback_entry), keys
// rebuilt from the leaf's partition bits.  Counts the windows it inserts.
// Leaves come here when they are large, which is where heavy hitters (one
// k-mer seen millions of times, Sec. II-B) end up: the lanes of a warp holding
// the same record (key and extension codes) add it once, with their number,
// so a hot key costs one atomic per warp instead of one per window.
template <int W>
__global__ void __launch_bounds__(256) records_insert_kernel(const Job j, const unsigned entry, HEntry<W>* t,
                                                             unsigned long long cap) {
    const Geometry g = j.g;
    const unsigned leaf = fallback_leaf(entry), rb = fallback_rb(entry), rs = fallback_rs(entry);
    const unsigned zb = g.zl_bits();
    const unsigned shift = (zb > g.p2 ? zb - g.p2 : 0u) - rb;
    const unsigned rmask = (1u << rb) - 1u;
    unsigned bucket;
    unsigned long long start, n;
    const unsigned long long* recs;
    if (g.p2 == 0) {
        bucket = leaf;
        start = j.l1_start[leaf];
        n = j.l1_fill[leaf];
        recs = j.l1_rec;
    } else {
        bucket = leaf >> g.p2;
        const unsigned sub = leaf & ((1u << g.p2) - 1u);
        start = j.l2_leaf_start ? j.l2_leaf_start[leaf]
                                : j.l2_base[bucket] + (unsigned long long)sub * j.l2_leafcap[bucket];
        n = j.l2_fill[leaf];
        recs = j.l2_rec;
    }
    unsigned windows = 0;
    bool stop = false;
    for (unsigned long long i0 = blockIdx.x * 256ull; i0 < n && !stop; i0 += (unsigned long long)gridDim.x * 256) {
        // the whole warp runs every iteration (lanes past the end or in another
        // range hold no record), so that it can compare its records
        const unsigned long long i = i0 + threadIdx.x;
        unsigned long long rec[W];
        bool have = i < n;
#pragma unroll
        for (int w = 0; w < W; ++w) rec[w] = have ? recs[(start + i) * W + w] : 0ull;
        const unsigned long long tail = rec[W - 1];
        if (have && rb && ((unsigned)((tail >> 6) >> shift) & rmask) != rs) have = false;  // another range
        // lanes with the same record: equal in every word (a lane without one
        // offers ~0, which no tail equals: a tail's low six bits are an
        // extension code, at most 36)
        unsigned peers = __match_any_sync(0xffffffffu, have ? tail : ~0ull);
#pragma unroll
        for (int w = 0; w < W - 1; ++w) peers &= __match_any_sync(0xffffffffu, rec[w]);
        const unsigned lane = threadIdx.x & 31;
        if (have && (peers & ((1u << lane) - 1u)) == 0) {  // the first lane of its group adds them all
            unsigned long long key[W];
#pragma unroll
            for (int w = 0; w < W - 1; ++w) key[w] = rec[w];
            const unsigned long long z = record_z(g, j.pass, j.bucket0 + bucket, tail);
            key[W - 1] = z_to_tail<W>(z, key, g.bt);
            const unsigned mult = __popc(peers);
            if (hbm_insert<W>(t, cap, key, z, ext_left(tail), ext_right(tail), j.status, mult)) windows += mult;
            else stop = true;
        }
        stop = __any_sync(0xffffffffu, stop);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) windows += __shfl_xor_sync(0xffffffffu, windows, o);
    if ((threadIdx.x & 31) == 0 && windows) atomicAdd(j.stats + 0, (unsigned long long)windows);
}

// Filter, classify and compact every occupied slot (one reservation per warp).
template <int W>
__global__ void __launch_bounds__(256) hbm_sweep_kernel(const Job j, const HEntry<W>* t, unsigned long long cap) {
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * 256;
    unsigned long long distinct = 0;
    for (unsigned long long base = blockIdx.x * 256ull + (threadIdx.x & ~31u); base < cap; base += stride) {
        const unsigned long long s = base + lane;
        const HEntry<W>* e = t + s;
        const unsigned long long k0 = s < cap ? e->key[0] : 0ull;
        const unsigned c = k0 ? e->count : 0u;
        const bool ok = k0 != 0ull && c >= j.min_count;
        distinct += k0 ? 1 : 0;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        unsigned long long wbase = 0;
        if (lane == 0 && m) wbase = atomicAdd(j.out_n, (unsigned long long)__popc(m));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (ok) {
            const unsigned long long pos = wbase + __popc(m & ((1u << lane) - 1u));
            if (pos < j.out_cap) {
                j.out_keys[pos * W] = k0 & ~(kOcc | kPub);
#pragma unroll
                for (int w = 1; w < W; ++w) j.out_keys[pos * W + w] = e->key[w];
                j.out_count[pos] = c;
                unsigned nl[4], nr[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) { nl[b] = e->ext[b]; nr[b] = e->ext[4 + b]; }
                uint4* eo = reinterpret_cast<uint4*>(j.out_ext + pos * 8);
                eo[0] = make_uint4(nl[0], nl[1], nl[2], nl[3]);
                eo[1] = make_uint4(nr[0], nr[1], nr[2], nr[3]);
                reinterpret_cast<uchar2*>(j.out_cls)[pos] =
                    make_uchar2(classify_side(nl, c, j), classify_side(nr, c, j));
            } else {
                atomicOr(j.status, ST_OUT_OVERFLOW);
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) distinct += __shfl_xor_sync(0xffffffffu, distinct, o);
    if (lane == 0 && distinct) atomicAdd(j.stats + 1, distinct);
}

static unsigned grid_for(unsigned long long items, int num_sms, unsigned per_sm) {
    unsigned long long g = (items + 255) / 256;
    const unsigned long long cap = (unsigned long long)num_sms * per_sm;
    if (g > cap) g = cap;
    return g ? (unsigned)g : 1u;
}

cudaError_t launch_direct_insert(const Job& j, void* table, unsigned long long cap, cudaStream_t s) {
    const unsigned long long grid = (j.n_reads + 255) / 256;
    if (grid == 0) return cudaSuccess;
    switch (j.g.W) {
        case 1: direct_insert_kernel<1><<<(unsigned)grid, 256, 0, s>>>(j, (HEntry<1>*)table, cap); break;
        case 2: direct_insert_kernel<2><<<(unsigned)grid, 256, 0, s>>>(j, (HEntry<2>*)table, cap); break;
        case 3: direct_insert_kernel<3><<<(unsigned)grid, 256, 0, s>>>(j, (HEntry<3>*)table, cap); break;
        case 4: direct_insert_kernel<4><<<(unsigned)grid, 256, 0, s>>>(j, (HEntry<4>*)table, cap); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_records_insert(const Job& j, unsigned entry, void* table, unsigned long long cap, int num_sms,
                                  cudaStream_t s) {
    const unsigned grid = (unsigned)num_sms * 4;
    switch (j.g.W) {
        case 1: records_insert_kernel<1><<<grid, 256, 0, s>>>(j, entry, (HEntry<1>*)table, cap); break;
        case 2: records_insert_kernel<2><<<grid, 256, 0, s>>>(j, entry, (HEntry<2>*)table, cap); break;
        case 3: records_insert_kernel<3><<<grid, 256, 0, s>>>(j, entry, (HEntry<3>*)table, cap); break;
        case 4: records_insert_kernel<4><<<grid, 256, 0, s>>>(j, entry, (HEntry<4>*)table, cap); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_hbm_sweep(const Job& j, const void* table, unsigned long long cap, int num_sms, cudaStream_t s) {
    const unsigned grid = grid_for(cap, num_sms, 8);
    switch (j.g.W) {
        case 1: hbm_sweep_kernel<1><<<grid, 256, 0, s>>>(j, (const HEntry<1>*)table, cap); break;
        case 2: hbm_sweep_kernel<2><<<grid, 256, 0, s>>>(j, (const HEntry<2>*)table, cap); break;
        case 3: hbm_sweep_kernel<3><<<grid, 256, 0, s>>>(j, (const HEntry<3>*)table, cap); break;
        case 4: hbm_sweep_kernel<4><<<grid, 256, 0, s>>>(j, (const HEntry<4>*)table, cap); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace kmer
