// Level-2 repartition: each level-1 bucket is split into 2^p2 leaves by the
// next bits of the mixed key, so that every leaf's distinct k-mers fit one
// CTA's shared-memory table.  Records move through shared memory in tiles
// and leave sorted by leaf (contiguous runs per warp).
#include "kernels.h"
#include "stage.cuh"

namespace kmer {

template <int W>
struct RepartShape {
    static constexpr unsigned S = W == 1 ? 4096 : (W == 2 ? 2048 : 1024);  // records per tile
};

__host__ __device__ inline unsigned repart_tile(unsigned W) {
    return W == 1 ? RepartShape<1>::S : (W == 2 ? RepartShape<2>::S : RepartShape<3>::S);
}

// One CTA: per bucket the records it really holds, its level-2 tile count and
// (uniform mode) the capacity of each of its leaves, then exclusive prefixes.
__global__ void __launch_bounds__(kStageThreads) l2_plan_kernel(const Job j, unsigned long long l2_capacity) {
    __shared__ unsigned long long warp_tmp[8];
    __shared__ unsigned long long s_tiles, s_slots;
    const unsigned P1 = 1u << j.g.p1, P2 = 1u << j.g.p2;
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

template <int W, unsigned MAXPER>
__global__ void __launch_bounds__(kStageThreads, 2) repart_kernel(const Job j) {
    constexpr unsigned S = RepartShape<W>::S;
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned P1 = 1u << j.g.p1, P2 = 1u << j.g.p2;
    StageBufs b = carve_stage(smem, W, S, P2);
    for (unsigned d = threadIdx.x; d < P2; d += kStageThreads) b.hist[d] = 0;
    __syncthreads();
    const unsigned zb = j.g.zl_bits();
    // the planner found the leaf layout larger than the buffer: write nothing, the host retries
    // (only the planner's bit: leaf overflows found by other CTAs must not stop the
    // counting, the host needs complete per-leaf totals for the exact layout)
    if (*(volatile unsigned*)j.status & ST_L2_PLAN) return;
    const unsigned long long total = j.tile_prefix[P1];
    for (unsigned long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        // bucket of this tile: last b with tile_prefix[b] <= tile
        unsigned lo = 0, hi = P1 - 1;
        while (lo < hi) {
            const unsigned mid = (lo + hi + 1) >> 1;
            if (j.tile_prefix[mid] <= tile) lo = mid; else hi = mid - 1;
        }
        const unsigned bucket = lo;
        const unsigned long long f = j.l1_fill[bucket], c = j.l1_cap[bucket];
        const unsigned long long n = f < c ? f : c;
        const unsigned long long begin = (tile - j.tile_prefix[bucket]) * S;
        const unsigned cnt = (unsigned)(n - begin < S ? n - begin : S);
        const unsigned long long* src = j.l1_rec + (j.l1_start[bucket] + begin) * W;
        // all of this thread's records of the tile are requested before any is used
        constexpr unsigned U = S / kStageThreads;
        unsigned long long rec[U][W];
#pragma unroll
        for (unsigned u = 0; u < U; ++u) {
            const unsigned e = u * kStageThreads + threadIdx.x;
#pragma unroll
            for (int w = 0; w < W; ++w) rec[u][w] = e < cnt ? __ldcs(src + (size_t)e * W + w) : 0ull;
        }
#pragma unroll
        for (unsigned u = 0; u < U; ++u) {
            const unsigned e = u * kStageThreads + threadIdx.x;
            unsigned m = 0xFFFFFFFFu;
            if (e < cnt) {
                const unsigned long long zl = rec[u][W - 1] >> 6;
                const unsigned sub = (unsigned)(zl >> (zb - j.g.p2)) & (P2 - 1u);
                const unsigned rank = atomicAdd(&b.hist[sub], 1u);
#pragma unroll
                for (int w = 0; w < W; ++w) b.stage[(size_t)e * W + w] = rec[u][w];
                m = (sub << 16) | rank;
            }
            b.meta[e] = m;
        }
        L2Dest dest{j.l2_fill, j.l2_leaf_start, j.l2_base[bucket], j.l2_leafcap[bucket], bucket << j.g.p2};
        flush_stage<W, MAXPER>(b, S, P2, dest, j.l2_rec, j.status, ST_L2_OVERFLOW);
    }
}

size_t repart_smem_bytes(unsigned W, unsigned p2) {
    return stage_smem_bytes(W, repart_tile(W), 1u << p2);
}

cudaError_t launch_l2_plan(const Job& j, unsigned long long l2_capacity, cudaStream_t s) {
    l2_plan_kernel<<<1, kStageThreads, 0, s>>>(j, l2_capacity);
    return cudaGetLastError();
}

template <int W, unsigned MAXPER>
static cudaError_t launch_repart_wp(const Job& j, int num_sms, cudaStream_t s) {
    const size_t smem = repart_smem_bytes(W, j.g.p2);
    cudaError_t e =
        cudaFuncSetAttribute(repart_kernel<W, MAXPER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    repart_kernel<W, MAXPER><<<num_sms * 2, kStageThreads, smem, s>>>(j);
    return cudaGetLastError();
}

template <int W>
static cudaError_t launch_repart_w(const Job& j, int num_sms, cudaStream_t s) {
    if ((1u << j.g.p2) <= 2 * kStageThreads) return launch_repart_wp<W, 2>(j, num_sms, s);
    return launch_repart_wp<W, kMaxStageDest / kStageThreads>(j, num_sms, s);
}

cudaError_t launch_repart(const Job& j, int num_sms, cudaStream_t s) {
    switch (j.g.W) {
        case 1: return launch_repart_w<1>(j, num_sms, s);
        case 2: return launch_repart_w<2>(j, num_sms, s);
        case 3: return launch_repart_w<3>(j, num_sms, s);
        case 4: return launch_repart_w<4>(j, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kmer
