// Steps a4-a7 fused: each leaf (partition) is counted in a shared-memory
// open-addressing table (the owner-local histogram of Sec. II-A use case 4,
// with the per-k-mer count and left/right extension tallies of Sec. II-B),
// then the table is swept once: k-mers below min_count are dropped, both
// sides are classified (Sec. II-C) and survivors are compacted to the output
// arrays.
//
// Persistent CTAs walk the leaves; while one leaf is being swept, the first
// batch of the next leaf's records is already loading into registers.
//
// Table (shared memory, planes of `cap_max` entries, a leaf uses the first
// `cap` slots): the tail word of each slot (0 = empty; record tail with the
// extension bits replaced by a mark bit; bit 0 = being published, W > 2
// only), W-1 head words (two-word keys keep tail and head side by side, one
// 16-byte pair per slot claimed by a 128-bit CAS, in probe groups of two
// slots), and nine 16-bit tallies packed in five 32-bit planes:
// left A, C, G, T, "no left extension" (so that count = sum of the five left
// lanes and needs no counter of its own), right A, C, G, T.  Slots are probed
// in groups of 32 bytes of keys (one read compares four tails, or two
// two-word keys).  A leaf with 65536 records or more (where a 16-bit tally
// could wrap) is recounted exactly by the HBM-table fallback; one whose keys
// do not fit its table is counted again in key ranges (leaf_split_kernel).
//
// Every plane is zero between leaves: the sweep clears each slot after
// reading it, so no separate clearing pass is needed.
#include "kernels.h"
#include "roll.cuh"

namespace kmer {

constexpr int kLeafThreads = 512;
constexpr int kLeafWarps = kLeafThreads / 32;
constexpr unsigned kLeafFull = 1u, kLeafTimeout = 4u;
constexpr unsigned kSpinLimit = 1u << 22;
constexpr unsigned kMaxGroupProbes = 16;  // 64 slots; a longer chain sends the leaf to the fallback
constexpr unsigned kLanePlanes = 5;
constexpr unsigned kMaxSubBits = 4;       // a leaf is split into at most 16 key ranges
// Slot tail of an occupied key: the record tail with its extension bits
// replaced by this mark; bit 0 marks a slot being published (W > 2).
constexpr unsigned long long kKeyMark = 32ull;
constexpr unsigned long long kBusy = 1ull;

template <int W>
struct LeafShape {
    static constexpr int U = W == 1 ? 4 : 2;  // records per thread per batch
    static constexpr int B = U * kLeafThreads;
};

// bytes per slot: tail, heads, 5 tally planes, survivor list entry
__host__ __device__ inline size_t leaf_slot_bytes(unsigned W) { return (size_t)8 * W + 4 * kLanePlanes + 4; }

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

struct Table {
    unsigned long long* tail;   // [cap_max]
    unsigned long long* heads;  // [(W-1) * cap_max]
    unsigned* lanes;            // [5 * cap_max]
    unsigned* list;             // [cap_max]
    unsigned stride;            // cap_max
};

// Two adjacent slots' tail words, re-read from shared memory on every call.
__device__ __forceinline__ ulonglong2 lds_v2_volatile(const unsigned long long* p) {
    ulonglong2 r;
    asm volatile("ld.volatile.shared.v2.u64 {%0, %1}, [%2];"
                 : "=l"(r.x), "=l"(r.y)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return r;
}

// Lane q in 0..8 lives in plane q >> 1, half q & 1.
__device__ __forceinline__ void bump(const Table& t, unsigned slot, unsigned q) {
    atomicAdd(&t.lanes[(q >> 1) * t.stride + slot], 1u << (16 * (q & 1)));
}

// Key words of a slot.  One-word keys: the tail plane.  Two-word keys:
// (tail, head) pairs, 16 bytes per slot over the first two planes, claimed
// whole by one 128-bit CAS.  Wider keys: the tail plane and W-1 head planes,
// published with a busy bit.
template <int W>
__device__ __forceinline__ unsigned long long& slot_tail(const Table& t, unsigned s) {
    return t.tail[W == 2 ? 2 * s : s];
}
template <int W>
__device__ __forceinline__ unsigned long long slot_head(const Table& t, unsigned w, unsigned s) {
    return W == 2 ? t.tail[2 * s + 1] : t.heads[(size_t)w * t.stride + s];
}
template <int W>
__device__ __forceinline__ void clear_key(const Table& t, unsigned s) {
    if (W == 2) {
        *reinterpret_cast<ulonglong2*>(t.tail + 2 * s) = make_ulonglong2(0ull, 0ull);
    } else {
        t.tail[s] = 0ull;  // head words of an empty slot are never read
    }
}
// Probe groups of a table of `cap` slots: 32 bytes of keys each.
template <int W>
__device__ __forceinline__ unsigned groups_of(unsigned cap) { return W == 2 ? cap / 2 : cap / 4; }

// 128-bit compare-and-swap on shared memory: {lo, hi} replaces {0, 0};
// returns the previous contents.
__device__ __forceinline__ void cas128_shared(unsigned long long* p, unsigned long long lo, unsigned long long hi,
                                              unsigned long long& old_lo, unsigned long long& old_hi) {
    asm volatile(
        "{\n\t.reg .b128 cmp, val, old;\n\t"
        "mov.b128 cmp, {%4, %4};\n\t"
        "mov.b128 val, {%2, %3};\n\t"
        "atom.shared.cas.b128 old, [%5], cmp, val;\n\t"
        "mov.b128 {%0, %1}, old;\n\t}"
        : "=l"(old_lo), "=l"(old_hi)
        : "l"(lo), "l"(hi), "l"(0ull), "r"((unsigned)__cvta_generic_to_shared(p))
        : "memory");
}

// Two-word keys: probe groups of two 16-byte slots.  A claim writes both
// words at once, but a plain 16-byte read may still see a slot being
// claimed with its tail and not yet its head; a tail match with another head
// is read again atomically (a CAS that can only fail) before it counts as a
// different key.
__device__ __forceinline__ int find_slot2(const Table& t, const unsigned long long ktail,
                                          const unsigned long long head, unsigned g, unsigned ngroups) {
    for (unsigned probe = 0; probe < 2 * kMaxGroupProbes; ++probe) {
        unsigned long long* grp = t.tail + 4 * g;
        const ulonglong2 a = lds_v2_volatile(grp);
        const ulonglong2 b = lds_v2_volatile(grp + 2);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            unsigned long long ct = s ? b.x : a.x, ch = s ? b.y : a.y;
            if (ct == 0ull) {  // empty (or still being claimed): try to claim it
                unsigned long long ot, oh;
                cas128_shared(grp + 2 * s, ktail, head, ot, oh);
                if (ot == 0ull && oh == 0ull) return (int)(2 * g + s);
                ct = ot;
                ch = oh;
            }
            if (ct != ktail) continue;
            if (ch != head) {
                unsigned long long ot, oh;
                cas128_shared(grp + 2 * s, 0ull, 0ull, ot, oh);  // the slot is claimed: no change, exact read
                if (ot != ktail || oh != head) continue;
            }
            return (int)(2 * g + s);
        }
        g = g + 1 == ngroups ? 0 : g + 1;
    }
    return -1;
}

template <int W>
__device__ __forceinline__ void insert_record(const Table& t, const unsigned long long (&rec)[W], unsigned ngroups,
                                              unsigned* s_flags) {
    const unsigned long long tail = rec[W - 1];
    const unsigned long long ktail = (tail & ~63ull) | kKeyMark;
    // home group from every in-leaf bit of z (for short keys the top bits of the
    // low word are partition bits, constant within a leaf): multiplicative hash
    const unsigned long long zl = tail >> 6;
    const unsigned hsh = (unsigned)((zl * 0x9E3779B97F4A7C15ull) >> 32);
    unsigned g = (unsigned)(((unsigned long long)hsh * ngroups) >> 32);
    int found = -1;
    if (W == 2) found = find_slot2(t, ktail, rec[0], g, ngroups);
    for (unsigned probe = 0; W != 2 && probe < kMaxGroupProbes && found < 0; ++probe) {
        unsigned long long* grp = t.tail + 4 * g;
        const ulonglong2 a = lds_v2_volatile(grp);
        const ulonglong2 b = lds_v2_volatile(grp + 2);
        unsigned long long cur[4] = {a.x, a.y, b.x, b.y};
        for (int s = 0; s < 4 && found < 0; ++s) {
            unsigned long long c = cur[s];
            if (c == 0ull) {  // first empty slot of the group: try to claim it
                const unsigned long long prev = atomicCAS(&grp[s], 0ull, W == 1 ? ktail : (ktail | kBusy));
                if (prev == 0ull) {
                    if (W > 1) {
#pragma unroll
                        for (int w = 0; w < W - 1; ++w) t.heads[(size_t)w * t.stride + 4 * g + s] = rec[w];
                        __threadfence_block();
                        atomicExch(&grp[s], ktail);
                    }
                    found = (int)(4 * g + s);
                    break;
                }
                c = prev;
            }
            if ((c & ~kBusy) != ktail) continue;
            if (W == 1) {
                found = (int)(4 * g + s);
                break;
            }
            unsigned spins = 0;
            while (c & kBusy) {
                if (++spins > kSpinLimit) {
                    atomicOr(s_flags, kLeafTimeout);
                    return;
                }
                c = *(volatile unsigned long long*)&grp[s];
            }
            __threadfence_block();
            bool same = true;
#pragma unroll
            for (int w = 0; w < W - 1; ++w)
                same = same && (*(volatile unsigned long long*)&t.heads[(size_t)w * t.stride + 4 * g + s] == rec[w]);
            if (same) found = (int)(4 * g + s);
        }
        g = g + 1 == ngroups ? 0 : g + 1;
    }
    if (found < 0) {
        atomicOr(s_flags, kLeafFull);
        return;
    }
    const unsigned l = ext_left(tail), r = ext_right(tail);
    bump(t, (unsigned)found, l ? l - 1 : 4u);  // every window has exactly one left lane
    if (r) bump(t, (unsigned)found, 4u + r);
}

// Clears slots [0, cap) of the table (all threads of the CTA).
template <int W>
__device__ __forceinline__ void clear_slots(const Table& t, unsigned cap) {
    for (unsigned s = threadIdx.x; s < cap; s += kLeafThreads) {
        clear_key<W>(t, s);
#pragma unroll
        for (unsigned p = 0; p < kLanePlanes; ++p) t.lanes[p * t.stride + s] = 0u;
    }
}

// Sweeps slots [0, cap): k-mers below min_count are dropped, survivors are
// classified and written (one output reservation per warp), and every slot
// is left clear.  Each warp takes a slice of cap / 16 slots.
template <int W>
__device__ __forceinline__ void sweep_table(const Job& j, const Table& t, const LeafInfo& li, unsigned cap,
                                            unsigned long long& distinct) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned cap_max = t.stride;
    const unsigned per = cap / kLeafWarps;  // a multiple of 32
    const unsigned s0 = wid * per;
    unsigned* mylist = t.list + s0;
    unsigned count = 0;
    for (unsigned s = s0 + lane; s < s0 + per; s += 32) {
        const unsigned long long tl = slot_tail<W>(t, s);
        const unsigned p0 = t.lanes[s], p1 = t.lanes[cap_max + s], p2 = t.lanes[2 * cap_max + s];
        const unsigned c = (p0 & 0xFFFFu) + (p0 >> 16) + (p1 & 0xFFFFu) + (p1 >> 16) + (p2 & 0xFFFFu);
        const bool ok = tl != 0ull && c >= j.min_count;
        distinct += tl != 0ull ? 1 : 0;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            mylist[count + __popc(m & ((1u << lane) - 1u))] = s;
        } else {
            clear_key<W>(t, s);
#pragma unroll
            for (unsigned p = 0; p < kLanePlanes; ++p) t.lanes[p * cap_max + s] = 0u;
        }
        count += __popc(m);
    }
    __syncwarp();
    unsigned long long wbase = 0;
    if (lane == 0 && count) wbase = atomicAdd(j.out_n, (unsigned long long)count);
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    for (unsigned i = lane; i < count; i += 32) {
        const unsigned s = mylist[i];
        const unsigned long long pos = wbase + i;
        const unsigned long long tl = slot_tail<W>(t, s);
        unsigned pl[kLanePlanes];
#pragma unroll
        for (unsigned p = 0; p < kLanePlanes; ++p) pl[p] = t.lanes[p * cap_max + s];
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W - 1; ++w) key[w] = slot_head<W>(t, w, s);
        clear_key<W>(t, s);
#pragma unroll
        for (unsigned p = 0; p < kLanePlanes; ++p) t.lanes[p * cap_max + s] = 0u;
        if (pos >= j.out_cap) {
            set_status(j, ST_OUT_OVERFLOW);
            continue;
        }
        const unsigned nl[4] = {pl[0] & 0xFFFFu, pl[0] >> 16, pl[1] & 0xFFFFu, pl[1] >> 16};
        const unsigned nr[4] = {pl[2] >> 16, pl[3] & 0xFFFFu, pl[3] >> 16, pl[4] & 0xFFFFu};
        const unsigned c = nl[0] + nl[1] + nl[2] + nl[3] + (pl[2] & 0xFFFFu);
        const unsigned long long z = record_z(j.g, j.pass, j.bucket0 + li.bucket, tl);
        key[W - 1] = z_to_tail<W>(z, key, j.g.bt);
#pragma unroll
        for (int w = 0; w < W; ++w) j.out_keys[pos * W + w] = key[w];
        j.out_count[pos] = c;
        uint4* eo = reinterpret_cast<uint4*>(j.out_ext + pos * 8);
        eo[0] = make_uint4(nl[0], nl[1], nl[2], nl[3]);
        eo[1] = make_uint4(nr[0], nr[1], nr[2], nr[3]);
        reinterpret_cast<uchar2*>(j.out_cls)[pos] = make_uchar2(classify_side(nl, c, j), classify_side(nr, c, j));
    }
}

// A leaf whose keys did not fit its table (and that has fewer than 65 536
// records): counted first as a whole in the whole table, then, if its keys
// still do not fit, in key ranges.  A range (rb, rs) holds the records whose
// next rb z bits below the leaf's bits equal rs; a range that does not fit is
// split in two, down to kMaxSubBits levels, in depth-first order, and a range
// that does not fit at the last level is handed to the HBM recount.  The
// table is clean on entry and on return.  Returns the windows this thread
// counted.
template <int W>
__device__ __forceinline__ unsigned count_in_ranges(const Job& j, const Table& t, const LeafInfo& li, unsigned leaf,
                                                 unsigned* s_flags, unsigned long long* distinct) {
    const unsigned long long n = li.n;
    const unsigned zb = j.g.zl_bits();
    const unsigned free_bits = zb > j.g.p2 ? zb - j.g.p2 : 0u;  // z bits below the leaf's
    const unsigned max_rb = free_bits < kMaxSubBits ? free_bits : kMaxSubBits;
    const unsigned cap = t.stride;
    const unsigned long long* src = li.recs + li.start * W;
    unsigned windows = 0;
    unsigned rb = 0, rs = 0;
    for (;;) {
        const unsigned shift = free_bits - rb, rmask = (1u << rb) - 1u;
        unsigned rwin = 0;
        for (unsigned long long i = threadIdx.x; i < n; i += kLeafThreads) {
            unsigned long long rec[W];
#pragma unroll
            for (int w = 0; w < W; ++w) rec[w] = src[i * W + w];
            if (((unsigned)((rec[W - 1] >> 6) >> shift) & rmask) != rs) continue;
            ++rwin;
            if (!*(volatile unsigned*)s_flags) insert_record<W>(t, rec, groups_of<W>(cap), s_flags);
        }
        __syncthreads();
        const unsigned flags = *(volatile unsigned*)s_flags;
        if (flags == kLeafFull && rb < max_rb) {  // split the range in two
            if (threadIdx.x == 0 && rb == 0) atomicAdd(j.stats + 3, 1ull);
            clear_slots<W>(t, cap);
            __syncthreads();
            if (threadIdx.x == 0) *s_flags = 0;
            __syncthreads();
            ++rb;
            rs <<= 1;
            continue;
        }
        if (flags) {
            if (threadIdx.x == 0) {
                if (flags & kLeafTimeout) {
                    set_status(j, ST_TIMEOUT);
                } else {  // exact recount of the range in HBM
                    const unsigned idx = atomicAdd(j.fb_n, 1u);
                    if (idx < j.fb_cap) j.fb_list[idx] = fallback_entry(leaf, rb, rs);
                    else set_status(j, ST_FALLBACK_FULL);
                }
            }
            clear_slots<W>(t, cap);
        } else {
            windows += rwin;
            sweep_table<W>(j, t, li, cap, *distinct);
        }
        __syncthreads();
        if (threadIdx.x == 0) *s_flags = 0;
        __syncthreads();
        // next range in depth-first order: climb while this range was a right half
        while (rb > 0 && (rs & 1u)) {
            rs >>= 1;
            --rb;
        }
        if (rb == 0) break;
        ++rs;
    }
    return windows;
}

// Leaves whose keys did not fit their table in leaf_kernel (the split list of
// each analysis), counted in key ranges.  Persistent CTAs over the listed
// leaves of every analysis; each analysis's list is complete when this
// kernel starts.
template <int W>
__global__ void __launch_bounds__(kLeafThreads, 2) leaf_split_kernel(const Job* __restrict__ jobs,
                                                                    const unsigned n_jobs, const unsigned cap_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_flags;
    const int lane = threadIdx.x & 31;
    Table t;
    t.stride = cap_max;
    t.tail = reinterpret_cast<unsigned long long*>(smem);
    t.heads = t.tail + cap_max;
    t.lanes = reinterpret_cast<unsigned*>(t.heads + (size_t)(W - 1) * cap_max);
    t.list = t.lanes + (size_t)kLanePlanes * cap_max;
    bool init = false;
    for (unsigned ji = 0; ji < n_jobs; ++ji) {
        const Job& j = jobs[ji];
        const unsigned n_split = *(volatile unsigned*)j.split_n;
        if (blockIdx.x >= n_split) continue;
        if (!init) {
            clear_slots<W>(t, cap_max);
            if (threadIdx.x == 0) s_flags = 0;
            __syncthreads();
            init = true;
        }
        unsigned long long windows = 0, distinct = 0;
        for (unsigned e = blockIdx.x; e < n_split; e += gridDim.x) {
            const unsigned leaf = j.split_list[e];
            const LeafInfo li = leaf_info(j, leaf);
            windows += count_in_ranges<W>(j, t, li, leaf, &s_flags, &distinct);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            windows += __shfl_xor_sync(0xffffffffu, windows, o);
            distinct += __shfl_xor_sync(0xffffffffu, distinct, o);
        }
        if (lane == 0 && windows) atomicAdd(j.stats + 0, windows);
        if (lane == 0 && distinct) atomicAdd(j.stats + 1, distinct);
    }
}

// Persistent CTAs over the leaves of every analysis of key width W; `leaf_off`
// is the exclusive prefix (n_jobs + 1) of the analyses' leaf counts.
template <int W>
__global__ void __launch_bounds__(kLeafThreads, 2) leaf_kernel(const Job* __restrict__ jobs,
                                                              const unsigned long long* __restrict__ leaf_off,
                                                              const unsigned n_jobs, const unsigned cap_max) {
    constexpr int U = LeafShape<W>::U, B = LeafShape<W>::B;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_flags;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long total = leaf_off[n_jobs];

    Table t;
    t.stride = cap_max;
    t.tail = reinterpret_cast<unsigned long long*>(smem);
    t.heads = t.tail + cap_max;
    t.lanes = reinterpret_cast<unsigned*>(t.heads + (size_t)(W - 1) * cap_max);
    t.list = t.lanes + (size_t)kLanePlanes * cap_max;
    for (unsigned s = threadIdx.x; s < cap_max; s += kLeafThreads) {
        clear_key<W>(t, s);
#pragma unroll
        for (unsigned p = 0; p < kLanePlanes; ++p) t.lanes[p * cap_max + s] = 0u;
    }
    if (threadIdx.x == 0) s_flags = 0;

    // statistics of the current analysis, added when the analysis changes
    unsigned long long windows = 0, distinct = 0;
    unsigned stat_job = 0;
    auto flush_stats = [&](unsigned ji) {
        unsigned long long d = distinct;
#pragma unroll
        for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0 && d) atomicAdd(jobs[ji].stats + 1, d);
        if (threadIdx.x == 0 && windows) atomicAdd(jobs[ji].stats + 0, windows);
        windows = distinct = 0;
    };

    unsigned long long g = blockIdx.x;
    unsigned ji = 0;
    unsigned leaf = 0;
    LeafInfo li;
    li.ok = false;
    unsigned long long batch[U][W];
    if (g < total) {
        ji = job_of(leaf_off, n_jobs, g);
        leaf = (unsigned)(g - leaf_off[ji]);
        li = leaf_info(jobs[ji], leaf);
        load_batch<W>(li, 0, batch);
        stat_job = ji;
    }
    __syncthreads();

    while (g < total) {
        const Job& j = jobs[ji];
        if (ji != stat_job) {
            flush_stats(stat_job);
            stat_job = ji;
        }
        const unsigned long long ng = g + gridDim.x;
        unsigned nji = ji, nleaf = 0;
        if (ng < total) {
            nji = job_of(leaf_off, n_jobs, ng);
            nleaf = (unsigned)(ng - leaf_off[nji]);
        }
        if (!li.ok || li.n >= 65536ull) {
            if (li.ok && threadIdx.x == 0) {  // 16-bit tallies could wrap: exact recount in HBM
                const unsigned idx = atomicAdd(j.fb_n, 1u);
                if (idx < j.fb_cap) j.fb_list[idx] = fallback_entry(leaf, 0, 0); else set_status(j, ST_FALLBACK_FULL);
            }
            g = ng;
            ji = nji;
            leaf = nleaf;
            li.ok = false;
            if (g < total) {
                li = leaf_info(jobs[ji], leaf);
                load_batch<W>(li, 0, batch);
            }
            continue;
        }
        // ---------------------------------------------------------- count
        const unsigned long long n = li.n;
        const unsigned long long want = ((n * j.table_ratio_num) >> 16) + 512;
        const unsigned cap = (unsigned)(want < cap_max ? ((want + 511) & ~511ull) : cap_max);
        const unsigned ngroups = groups_of<W>(cap);
        for (unsigned long long first = 0; first < n; first += B) {
            if (first) load_batch<W>(li, first, batch);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const unsigned long long i = first + (unsigned long long)u * kLeafThreads + threadIdx.x;
                if (i < n && !*(volatile unsigned*)&s_flags) insert_record<W>(t, batch[u], ngroups, &s_flags);
            }
        }
        __syncthreads();
        const unsigned flags = s_flags;
        // the next leaf's first batch loads while this one is swept
        LeafInfo nli;
        nli.ok = false;
        if (ng < total) {
            nli = leaf_info(jobs[nji], nleaf);
            load_batch<W>(nli, 0, batch);
        }
        const unsigned per = cap / kLeafWarps;  // a multiple of 32
        const unsigned s0 = wid * per;
        if (flags) {
            if (threadIdx.x == 0) {
                if (flags & kLeafTimeout) {
                    set_status(j, ST_TIMEOUT);
                } else {  // keys did not fit: counted again, in key ranges (leaf_split_kernel)
                    const unsigned idx = atomicAdd(j.split_n, 1u);
                    if (idx < j.split_cap) {
                        j.split_list[idx] = leaf;
                    } else {
                        const unsigned f = atomicAdd(j.fb_n, 1u);
                        if (f < j.fb_cap) j.fb_list[f] = fallback_entry(leaf, 0, 0);
                        else set_status(j, ST_FALLBACK_FULL);
                    }
                }
            }
            for (unsigned s = s0 + lane; s < s0 + per; s += 32) {  // leave the table clean
                clear_key<W>(t, s);
#pragma unroll
                for (unsigned p = 0; p < kLanePlanes; ++p) t.lanes[p * cap_max + s] = 0u;
            }
        } else {
            if (threadIdx.x == 0) windows += n;
            sweep_table<W>(j, t, li, cap, distinct);  // filter, classify, compact (per warp)
        }
        if (threadIdx.x == 0) s_flags = 0;
        __syncthreads();  // the clean table is reused by the next leaf
        g = ng;
        ji = nji;
        leaf = nleaf;
        li = nli;
    }
    if (blockIdx.x < total) flush_stats(stat_job);
}

template <int W>
static cudaError_t launch_leaf_w(const Job* jobs, const unsigned long long* leaf_off, unsigned n_jobs,
                                 unsigned long long leaves, unsigned cap_max, int num_sms, cudaStream_t s) {
    const size_t smem = leaf_smem_bytes(W, cap_max);
    cudaError_t e = raise_smem_limit((const void*)leaf_kernel<W>, smem);
    if (e != cudaSuccess) return e;
    unsigned long long grid = (unsigned long long)num_sms * 2;
    if (grid > leaves) grid = leaves;
    if (grid == 0) return cudaSuccess;
    leaf_kernel<W><<<(unsigned)grid, kLeafThreads, smem, s>>>(jobs, leaf_off, n_jobs, cap_max);
    return cudaGetLastError();
}

template <int W>
static cudaError_t launch_leaf_split_w(const Job* jobs, unsigned n_jobs, unsigned cap_max, int num_sms,
                                       cudaStream_t s) {
    const size_t smem = leaf_smem_bytes(W, cap_max);
    cudaError_t e =
        raise_smem_limit((const void*)leaf_split_kernel<W>, smem);
    if (e != cudaSuccess) return e;
    if (n_jobs == 0) return cudaSuccess;
    leaf_split_kernel<W><<<(unsigned)num_sms * 2, kLeafThreads, smem, s>>>(jobs, n_jobs, cap_max);
    return cudaGetLastError();
}

cudaError_t launch_leaf_split(unsigned W, const Job* jobs, unsigned n_jobs, unsigned cap_max, int num_sms,
                              cudaStream_t s) {
    switch (W) {
        case 1: return launch_leaf_split_w<1>(jobs, n_jobs, cap_max, num_sms, s);
        case 2: return launch_leaf_split_w<2>(jobs, n_jobs, cap_max, num_sms, s);
        case 3: return launch_leaf_split_w<3>(jobs, n_jobs, cap_max, num_sms, s);
        case 4: return launch_leaf_split_w<4>(jobs, n_jobs, cap_max, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_leaf(unsigned W, const Job* jobs, const unsigned long long* leaf_off, unsigned n_jobs,
                        unsigned long long leaves, unsigned cap_max, int num_sms, cudaStream_t s) {
    switch (W) {
        case 1: return launch_leaf_w<1>(jobs, leaf_off, n_jobs, leaves, cap_max, num_sms, s);
        case 2: return launch_leaf_w<2>(jobs, leaf_off, n_jobs, leaves, cap_max, num_sms, s);
        case 3: return launch_leaf_w<3>(jobs, leaf_off, n_jobs, leaves, cap_max, num_sms, s);
        case 4: return launch_leaf_w<4>(jobs, leaf_off, n_jobs, leaves, cap_max, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kmer
