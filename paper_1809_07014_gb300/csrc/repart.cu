// Level-2 repartition: each level-1 bucket is split into 2^p2 leaves by the
// next bits of the mixed key, so that every leaf's distinct k-mers fit one
// CTA's shared-memory table.  Records move through shared memory in tiles
// and leave sorted by leaf (contiguous runs per warp).
#include "kernels.h"
#include "stage.cuh"

namespace kmer {

constexpr unsigned kRepartThreads = 512;

template <int W>
struct RepartShape {
    static constexpr unsigned S = W == 1 ? 4096 : 2048;  // records per tile
};

__host__ __device__ inline unsigned repart_tile(unsigned W) {
    return W == 1 ? RepartShape<1>::S : (W == 2 ? RepartShape<2>::S : RepartShape<3>::S);
}

// One CTA per analysis: per bucket the records it really holds, its level-2
// tile count and (uniform mode) the capacity of each of its leaves, then
// exclusive prefixes.
__global__ void __launch_bounds__(kStageThreads) l2_plan_kernel(const Job* __restrict__ jobs) {
    const Job& j = jobs[blockIdx.x];
    if (j.g.p2 == 0) return;
    const unsigned long long l2_capacity = j.l2_capacity;
    __shared__ unsigned long long warp_tmp[8];
    __shared__ unsigned long long s_tiles, s_slots;
    const unsigned P1 = job_buckets(j), P2 = 1u << j.g.p2;
    const unsigned tile = repart_tile(j.g.W);
    if (threadIdx.x == 0) { s_tiles = 0; s_slots = 0; }
    __syncthreads();
    for (unsigned base = 0; base < P1; base += kStageThreads) {
        const unsigned b = base + threadIdx.x;
        unsigned long long n = 0, tiles = 0, slots = 0;
        unsigned leafcap = 0;
        if (b < P1) {
            const unsigned long long f = j.l1_fill[b], c = j.l1_cap[b];
            n = f < c ? f : c;
            tiles = (n + tile - 1) / tile;
            const unsigned long long mean = (n + P2 - 1) / P2;
            const unsigned long long lc = n ? (mean * j.l2_slack_num >> 8) + 256 : 0;
            leafcap = lc > 0xFFFFFFF0ull ? 0xFFFFFFF0u : (unsigned)lc;
            slots = (unsigned long long)leafcap * P2;
        }
        unsigned long long tot_t, tot_s;
        const unsigned long long ex_t = block_scan_u64(tiles, warp_tmp, &tot_t);
        const unsigned long long ex_s = block_scan_u64(slots, warp_tmp, &tot_s);
        if (b < P1) {
            j.tile_prefix[b] = s_tiles + ex_t;
            j.l2_leafcap[b] = leafcap;
            j.l2_base[b] = s_slots + ex_s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_tiles += tot_t;
            s_slots += tot_s;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        j.tile_prefix[P1] = s_tiles;
        if (s_slots > l2_capacity) atomicOr(j.status, ST_L2_OVERFLOW | ST_L2_PLAN);
    }
}

struct L2Dest {
    unsigned long long* fill;         // per leaf
    const unsigned long long* exact;  // per leaf + 1 (exact mode) or null
    unsigned long long base;          // uniform mode: first record index of the bucket's leaves
    unsigned leafcap;                 // uniform mode
    unsigned leaf0;                   // bucket << p2
    __device__ unsigned long long reserve(unsigned d, unsigned n) {
        return atomicAdd(fill + leaf0 + d, (unsigned long long)n);
    }
    __device__ unsigned long long start(unsigned d) const {
        return exact ? __ldg(exact + leaf0 + d) : base + (unsigned long long)d * leafcap;
    }
    __device__ unsigned long long cap(unsigned d) const {
        return exact ? __ldg(exact + leaf0 + d + 1) - __ldg(exact + leaf0 + d) : (unsigned long long)leafcap;
    }
};

// Level-2 tiles of every analysis before analysis i (one CTA).
__global__ void __launch_bounds__(kStageThreads) job_tiles_kernel(const Job* __restrict__ jobs, const unsigned n_jobs,
                                                                   unsigned long long* __restrict__ job_tile_off) {
    __shared__ unsigned long long warp_tmp[8];
    __shared__ unsigned long long s_run;
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (unsigned base = 0; base < n_jobs; base += kStageThreads) {
        const unsigned i = base + threadIdx.x;
        unsigned long long t = 0;
        if (i < n_jobs) {
            const Job& jb = jobs[i];
            // an analysis whose planner overflowed contributes no tiles (the host retries it)
            if (jb.g.p2 && !(*(volatile unsigned*)jb.status & ST_L2_PLAN)) t = jb.tile_prefix[job_buckets(jb)];
        }
        unsigned long long tot;
        const unsigned long long ex = block_scan_u64(t, warp_tmp, &tot);
        if (i < n_jobs) job_tile_off[i] = s_run + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_run += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) job_tile_off[n_jobs] = s_run;
}

// Where one level-2 tile's records are: its analysis, bucket and record range.
struct RepartTile {
    unsigned ji, bucket, cnt;
    const unsigned long long* src;
};

// A CTA's tiles come in increasing order, gridDim.x apart, and a bucket spans
// many tiles: the bucket of the next tile is the previous one or the one
// after it, found with one or two loads; a search (a chain of dependent
// loads, each an L2 round trip) is needed only on a CTA's first tile of an
// analysis or after a jump over several buckets.
struct TileCursor {
    unsigned ji = 0xFFFFFFFFu, bucket = 0;
};

__device__ __forceinline__ RepartTile repart_tile_at(const Job* __restrict__ jobs,
                                                     const unsigned long long* __restrict__ job_tile_off,
                                                     const unsigned n_jobs, const unsigned long long gt,
                                                     const unsigned S, TileCursor& cur) {
    RepartTile rt;
    if (cur.ji == 0xFFFFFFFFu || (cur.ji + 1 < n_jobs && job_tile_off[cur.ji + 1] <= gt)) {
        cur.ji = job_of(job_tile_off, n_jobs, gt);
        cur.bucket = 0xFFFFFFFFu;
    }
    rt.ji = cur.ji;
    const Job& j = jobs[rt.ji];
    const unsigned long long tile = gt - job_tile_off[rt.ji];
    const unsigned last = job_buckets(j) - 1;
    // bucket of this tile: last b with tile_prefix[b] <= tile
    unsigned b = cur.bucket;
    if (b != 0xFFFFFFFFu && b < last && j.tile_prefix[b + 1] <= tile) {
        ++b;
        if (b < last && j.tile_prefix[b + 1] <= tile) b = 0xFFFFFFFFu;  // more than one bucket ahead
    }
    if (b == 0xFFFFFFFFu) {
        unsigned lo = cur.bucket == 0xFFFFFFFFu ? 0 : cur.bucket, hi = last;
        while (lo < hi) {
            const unsigned mid = (lo + hi + 1) >> 1;
            if (j.tile_prefix[mid] <= tile) lo = mid; else hi = mid - 1;
        }
        b = lo;
    }
    cur.bucket = b;
    rt.bucket = b;
    const unsigned lo = b;
    const unsigned long long f = j.l1_fill[lo], c = j.l1_cap[lo];
    const unsigned long long n = f < c ? f : c;
    const unsigned long long begin = (tile - j.tile_prefix[lo]) * S;
    rt.cnt = (unsigned)(n - begin < S ? n - begin : S);
    rt.src = j.l1_rec + (j.l1_start[lo] + begin) * j.g.W;
    return rt;
}

// Persistent CTAs over the level-2 tiles of every analysis (records of three
// or four words; narrower records take repart_tma_kernel below).  A tile's
// records are requested (into registers) before the previous tile is
// flushed, so the loads overlap the flush.  Shared memory is laid out for
// `pmax` leaves per bucket, the largest fan-out of the launch.
template <int W, unsigned MAXPER>
__global__ void __launch_bounds__(kRepartThreads, 2) repart_kernel(const Job* __restrict__ jobs,
                                                                 const unsigned long long* __restrict__ job_tile_off,
                                                                 const unsigned n_jobs, const unsigned pmax) {
    constexpr unsigned S = RepartShape<W>::S;
    constexpr unsigned U = S / kRepartThreads;
    extern __shared__ __align__(16) unsigned char smem[];
    const StageBufs b = carve_stage(smem, W, S, pmax);
    for (unsigned d = threadIdx.x; d < pmax; d += kRepartThreads) b.hist[d] = 0;
    const unsigned long long all = job_tile_off[n_jobs];
    unsigned long long gt = blockIdx.x;
    unsigned long long rec[U][W];
    RepartTile rt{};
    TileCursor cur;
    auto load = [&](const RepartTile& x) {
#pragma unroll
        for (unsigned u = 0; u < U; ++u) {
            const unsigned e = u * kRepartThreads + threadIdx.x;
#pragma unroll
            for (int w = 0; w < W; ++w) rec[u][w] = e < x.cnt ? __ldcs(x.src + (size_t)e * W + w) : 0ull;
        }
    };
    if (gt < all) {
        rt = repart_tile_at(jobs, job_tile_off, n_jobs, gt, S, cur);
        load(rt);
    }
    __syncthreads();
    while (gt < all) {
        const Job& j = jobs[rt.ji];
        const unsigned P2 = 1u << j.g.p2;
        const unsigned zb = j.g.zl_bits();
        const unsigned shift = zb - j.g.p2;
        unsigned m[U];
#pragma unroll
        for (unsigned u = 0; u < U; ++u) {
            const unsigned e = u * kRepartThreads + threadIdx.x;
            m[u] = 0xFFFFFFFFu;
            if (e < rt.cnt) {
                const unsigned long long zl = rec[u][W - 1] >> 6;
                const unsigned sub = (unsigned)(zl >> shift) & (P2 - 1u);
                const unsigned rank = atomicAdd(&b.hist[sub], 1u);
#pragma unroll
                for (int w = 0; w < W; ++w) b.stage[(size_t)e * W + w] = rec[u][w];
                m[u] = (sub << 16) | rank;
            }
        }
        // the next tile's loads are in flight during this tile's flush
        const unsigned long long ngt = gt + gridDim.x;
        RepartTile nrt{};
        if (ngt < all) {
            nrt = repart_tile_at(jobs, job_tile_off, n_jobs, ngt, S, cur);
            load(nrt);
        }
        L2Dest dest{j.l2_fill, j.l2_leaf_start, j.l2_base[rt.bucket], j.l2_leafcap[rt.bucket], rt.bucket << j.g.p2};
        flush_stage_regs<W, MAXPER, L2Dest, kRepartThreads, U>(b, S, P2, dest, j.l2_rec, j.status, ST_L2_OVERFLOW, m);
        gt = ngt;
        rt = nrt;
    }
}

// ------------------------------------------------------------------------
// One- and two-word records: tiles arrive by bulk asynchronous copies (the TMA engine,
// cp.async.bulk completing on an mbarrier) into two shared-memory buffers, two
// tiles ahead of the one being flushed, so no registers hold records in
// flight and the flush reads each record straight from the tile buffer.
constexpr unsigned kTmaWaitLimit = 1u << 20;  // try_wait rounds before a wait gives up

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase `phase` of an mbarrier to complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase) {
    for (unsigned i = 0; i < kTmaWaitLimit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// One thread: announce `bytes` on the barrier and start the bulk copy
// (both addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Records of a tile sit `lead` records into its buffer: the copy starts at
// the 16-byte boundary at or below the tile's first record (the level-1
// region is 256-byte aligned and padded at its end, so the rounded range
// stays inside it).
__device__ __forceinline__ unsigned tile_lead(const RepartTile& rt) {
    return (unsigned)(reinterpret_cast<unsigned long long>(rt.src) & 15ull) >> 3;
}

template <int W>
__device__ __forceinline__ void issue_tile(const RepartTile& rt, unsigned long long* buf, unsigned long long* bar) {
    const unsigned lead = tile_lead(rt);
    const unsigned bytes = ((lead + rt.cnt * W) * 8u + 15u) & ~15u;
    bulk_load(buf, rt.src - lead, bytes, bar);
}

// Shared memory: two tile buffers (each a tile plus 16 bytes of lead), two
// mbarriers, then the staging arrays without a meta array.
__host__ __device__ inline size_t repart_tma_smem_bytes(unsigned W, unsigned pmax) {
    const size_t S = W == 1 ? RepartShape<1>::S : RepartShape<2>::S;
    return 2 * (S * W + 2) * 8 + 16 + (size_t)pmax * 8 + 3 * (size_t)pmax * 4 + S * 4 + 128;
}

// A tile buffer's state: the tile it holds or is receiving, whether a copy
// into it is still unwaited, and the barrier phase that copy completes.
struct TmaSlot {
    RepartTile rt;
    bool pending;
    unsigned phase;
};

template <int W, unsigned MAXPER>
__global__ void __launch_bounds__(kRepartThreads, 2) repart_tma_kernel(const Job* __restrict__ jobs,
                                                                     const unsigned long long* __restrict__ job_tile_off,
                                                                     const unsigned n_jobs, const unsigned pmax) {
    static_assert(W <= 2, "tile buffers sized for one- and two-word records");
    constexpr unsigned S = RepartShape<W>::S, U = S / kRepartThreads;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* const buf0 = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* const buf1 = buf0 + S * W + 2;
    unsigned long long* const bar = buf1 + S * W + 2;  // two mbarriers
    StageBufs sb;
    sb.stage = nullptr;
    sb.meta = nullptr;
    sb.wbase = bar + 2;
    sb.ok_end = reinterpret_cast<unsigned*>(sb.wbase + pmax);
    sb.hist = sb.ok_end + pmax;
    sb.lbase = sb.hist + pmax;
    sb.order = sb.lbase + pmax;
    sb.warp_tmp = sb.order + S;
    for (unsigned d = threadIdx.x; d < pmax; d += kRepartThreads) sb.hist[d] = 0;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    const unsigned long long all = job_tile_off[n_jobs];
    TileCursor cur;
    TmaSlot s0{{}, false, 0}, s1{{}, false, 0};
    auto start = [&](TmaSlot& sl, unsigned long long* bf, unsigned long long* br, unsigned long long g) {
        sl.rt = repart_tile_at(jobs, job_tile_off, n_jobs, g, S, cur);
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile<W>(sl.rt, bf, br);
        }
        sl.pending = true;
    };
    // waits for the slot's tile, flushes it, and refills the slot with the
    // tile two steps ahead; false after a wait that gave up
    auto run = [&](TmaSlot& sl, unsigned long long* bf, unsigned long long* br, unsigned long long gt) -> bool {
        const RepartTile t = sl.rt;
        const Job& j = jobs[t.ji];
        if (!mbar_wait(br, sl.phase)) {
            if (threadIdx.x == 0) set_status(j, ST_TIMEOUT);
            return false;
        }
        sl.pending = false;
        sl.phase ^= 1u;
        const unsigned long long* tile = bf + tile_lead(t);
        const unsigned P2 = 1u << j.g.p2;
        const unsigned shift = j.g.zl_bits() - j.g.p2;
        unsigned m[U];
#pragma unroll
        for (unsigned u = 0; u < U; ++u) {
            const unsigned e = u * kRepartThreads + threadIdx.x;
            m[u] = 0xFFFFFFFFu;
            if (e < t.cnt) {
                const unsigned sub = (unsigned)((tile[(size_t)e * W + W - 1] >> 6) >> shift) & (P2 - 1u);
                m[u] = (sub << 16) | atomicAdd(&sb.hist[sub], 1u);
            }
        }
        StageBufs b = sb;
        b.stage = const_cast<unsigned long long*>(tile);
        L2Dest dest{j.l2_fill, j.l2_leaf_start, j.l2_base[t.bucket], j.l2_leafcap[t.bucket], t.bucket << j.g.p2};
        flush_stage_regs<W, MAXPER, L2Dest, kRepartThreads, U>(b, S, P2, dest, j.l2_rec, j.status, ST_L2_OVERFLOW, m);
        // the flush ends on a barrier: every thread is done with this buffer
        const unsigned long long g2 = gt + 2ull * gridDim.x;
        if (g2 < all) start(sl, bf, br, g2);
        return true;
    };
    if (blockIdx.x < all) start(s0, buf0, &bar[0], blockIdx.x);
    if (blockIdx.x + (unsigned long long)gridDim.x < all) start(s1, buf1, &bar[1], blockIdx.x + gridDim.x);
    for (unsigned long long gt = blockIdx.x; gt < all; gt += 2ull * gridDim.x) {
        if (!run(s0, buf0, &bar[0], gt)) break;
        if (gt + gridDim.x >= all) break;
        if (!run(s1, buf1, &bar[1], gt + gridDim.x)) break;
    }
    // after a wait that gave up: no copy may still be writing this CTA's shared memory
    if (s0.pending) mbar_wait(&bar[0], s0.phase);
    if (s1.pending) mbar_wait(&bar[1], s1.phase);
}

size_t repart_smem_bytes(unsigned W, unsigned p2) {
    return W <= 2 ? repart_tma_smem_bytes(W, 1u << p2) : stage_smem_bytes(W, repart_tile(W), 1u << p2);
}

cudaError_t launch_l2_plan(const Job* jobs, unsigned n_jobs, unsigned long long* job_tile_off, cudaStream_t s) {
    if (n_jobs == 0) return cudaSuccess;
    l2_plan_kernel<<<n_jobs, kStageThreads, 0, s>>>(jobs);
    job_tiles_kernel<<<1, kStageThreads, 0, s>>>(jobs, n_jobs, job_tile_off);
    return cudaGetLastError();
}

template <int W, unsigned MAXPER>
static cudaError_t launch_repart_wp(const Job* jobs, const unsigned long long* job_tile_off, unsigned n_jobs,
                                    unsigned max_p2, int num_sms, cudaStream_t s) {
    const size_t smem = repart_smem_bytes(W, max_p2);
    cudaError_t e =
        raise_smem_limit((const void*)repart_kernel<W, MAXPER>, smem);
    if (e != cudaSuccess) return e;
    repart_kernel<W, MAXPER><<<num_sms * 2, kRepartThreads, smem, s>>>(jobs, job_tile_off, n_jobs, 1u << max_p2);
    return cudaGetLastError();
}

template <int W, unsigned MAXPER>
static cudaError_t launch_repart_tma(const Job* jobs, const unsigned long long* job_tile_off, unsigned n_jobs,
                                     unsigned max_p2, int num_sms, cudaStream_t s) {
    const size_t smem = repart_tma_smem_bytes(W, 1u << max_p2);
    cudaError_t e =
        raise_smem_limit((const void*)repart_tma_kernel<W, MAXPER>, smem);
    if (e != cudaSuccess) return e;
    repart_tma_kernel<W, MAXPER><<<num_sms * 2, kRepartThreads, smem, s>>>(jobs, job_tile_off, n_jobs, 1u << max_p2);
    return cudaGetLastError();
}

template <int W>
static cudaError_t launch_repart_w(const Job* jobs, const unsigned long long* job_tile_off, unsigned n_jobs,
                                   unsigned max_p2, int num_sms, cudaStream_t s) {
    if constexpr (W <= 2) {
        if ((1u << max_p2) <= 2 * kRepartThreads)
            return launch_repart_tma<W, 2>(jobs, job_tile_off, n_jobs, max_p2, num_sms, s);
        return launch_repart_tma<W, kMaxStageDest / kRepartThreads>(jobs, job_tile_off, n_jobs, max_p2, num_sms, s);
    } else {
        if ((1u << max_p2) <= 2 * kRepartThreads)
            return launch_repart_wp<W, 2>(jobs, job_tile_off, n_jobs, max_p2, num_sms, s);
        return launch_repart_wp<W, kMaxStageDest / kRepartThreads>(jobs, job_tile_off, n_jobs, max_p2, num_sms, s);
    }
}

cudaError_t launch_repart(unsigned W, const Job* jobs, const unsigned long long* job_tile_off, unsigned n_jobs,
                          unsigned max_p2, int num_sms, cudaStream_t s) {
    switch (W) {
        case 1: return launch_repart_w<1>(jobs, job_tile_off, n_jobs, max_p2, num_sms, s);
        case 2: return launch_repart_w<2>(jobs, job_tile_off, n_jobs, max_p2, num_sms, s);
        case 3: return launch_repart_w<3>(jobs, job_tile_off, n_jobs, max_p2, num_sms, s);
        case 4: return launch_repart_w<4>(jobs, job_tile_off, n_jobs, max_p2, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kmer
