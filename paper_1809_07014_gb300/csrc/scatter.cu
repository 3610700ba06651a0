// Level-1 scatter: one thread per read rolls its k-windows (a2, a3), turns
// each into a W-word record and hands it to the level-1 bucket picked by the
// top bits of the mixed key.  This is the all-to-all k-mer exchange of the
// paper's k-mer analysis (Sec. II-B), done as a device-wide partition in HBM:
// a bucket plays the role of the owning processor.
#include "kernels.h"
#include "roll.cuh"
#include "stage.cuh"

namespace kmer {

template <int W>
struct ScatterShape {
    // read positions per round: 4096 records (W = 1) or about 48 KB of records staged
    static constexpr unsigned R = W == 1 ? 16 : (W == 2 ? 12 : (W == 3 ? 8 : 6));
    static constexpr unsigned S = R * kStageThreads;                 // staged records per round
};

struct L1Dest {
    unsigned long long* fill;
    const unsigned long long* startp;
    const unsigned long long* capp;
    __device__ unsigned long long reserve(unsigned d, unsigned n) { return atomicAdd(fill + d, (unsigned long long)n); }
    __device__ unsigned long long start(unsigned d) const { return __ldg(startp + d); }
    __device__ unsigned long long cap(unsigned d) const { return __ldg(capp + d); }
};

// One CTA: 256 consecutive reads of job j (a read tile).
// MAXPER: destinations handled by one thread in a flush (fan-out / 256).
template <int W, unsigned MAXPER, bool HI, bool GATE>
__device__ __forceinline__ void scatter_tile(const Job& j, const unsigned long long r0, const unsigned long long r1,
                                             unsigned char* smem) {
    constexpr unsigned R = ScatterShape<W>::R, S = ScatterShape<W>::S;
    __shared__ unsigned s_maxlen;
    const unsigned P = 1u << j.g.p1;
    StageBufs b = carve_stage(smem, W, S, P);
    if (threadIdx.x == 0) s_maxlen = 0;
    for (unsigned d = threadIdx.x; d < P; d += kStageThreads) b.hist[d] = 0;
    __syncthreads();

    const unsigned long long r = r0 + threadIdx.x;
    Roll<W, HI> roll;
    unsigned L = 0;  // reads are shorter than 2^31 bases
    const bool have = r < r1;
    if (have) {
        roll.init(j, r);
        L = (unsigned)roll.L;
        atomicMax(&s_maxlen, (unsigned)L);
    }
    __syncthreads();
    const unsigned rounds = (s_maxlen + R) / R;  // steps 0 .. maxlen
    L1Dest dest{j.l1_fill, j.l1_start, j.l1_cap};
    const Geometry g = j.g;
    const unsigned pass = j.pass;
    const unsigned long long* gate = j.gate;  // Bloom gate (GATE): emit only keys in F2
    const unsigned gate_bits = j.gate_bits;
    unsigned emitted = 0;
    for (unsigned round = 0; round < rounds; ++round) {
#pragma unroll 2
        for (unsigned s = 0; s < R; ++s) {
            const unsigned t = round * R + s;
            const unsigned e = s * kStageThreads + threadIdx.x;
            unsigned m = 0xFFFFFFFFu;
            if (have && t <= L) {
                unsigned long long key[W], rec[W];
                unsigned lc = 0, rc = 0, bucket = 0;
                if (roll.step(t, key, lc, rc) && (!GATE || gate_has<W>(gate, gate_bits, key)) &&
                    make_record<W>(g, pass, key, lc, rc, rec, bucket)) {
                    const unsigned rank = atomicAdd(&b.hist[bucket], 1u);
#pragma unroll
                    for (int w = 0; w < W; ++w) b.stage[(size_t)e * W + w] = rec[w];
                    m = (bucket << 16) | rank;
                    ++emitted;
                }
            }
            b.meta[e] = m;
        }
        flush_stage<W, MAXPER>(b, S, P, dest, j.l1_rec, j.status, ST_L1_OVERFLOW);
    }
    // windows emitted into this pass (checked against the windows the leaves count)
#pragma unroll
    for (int o = 16; o; o >>= 1) emitted += __shfl_xor_sync(0xffffffffu, emitted, o);
    if ((threadIdx.x & 31) == 0 && emitted) atomicAdd(j.stats + 2, (unsigned long long)emitted);
}

// One CTA per read tile over all jobs (all of key width W).
template <int W, unsigned MAXPER, bool HI, bool GATE>
__global__ void __launch_bounds__(kStageThreads, W == 1 ? 3 : 2)
scatter_kernel(const Job* __restrict__ jobs, const unsigned long long* __restrict__ tile_off, const unsigned n_jobs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned long long t = blockIdx.x;
    const unsigned ji = job_of(tile_off, n_jobs, t);
    const Job& j = jobs[ji];
    const unsigned long long r0 = (t - tile_off[ji]) * kStageThreads;
    const unsigned long long r1 = r0 + kStageThreads < j.n_reads ? r0 + kStageThreads : j.n_reads;
    scatter_tile<W, MAXPER, HI, GATE>(j, r0, r1, smem);
}

size_t scatter_smem_bytes(unsigned W, unsigned p1) {
    const unsigned P = 1u << p1;
    switch (W) {
        case 1: return stage_smem_bytes(1, ScatterShape<1>::S, P);
        case 2: return stage_smem_bytes(2, ScatterShape<2>::S, P);
        case 3: return stage_smem_bytes(3, ScatterShape<3>::S, P);
        default: return stage_smem_bytes(4, ScatterShape<4>::S, P);
    }
}

template <int W, unsigned MAXPER, bool HI, bool GATE>
static cudaError_t launch_scatter_wpg(const Job* jobs, const unsigned long long* tile_off, unsigned n_jobs,
                                      unsigned long long tiles, unsigned max_p1, cudaStream_t s) {
    const size_t smem = scatter_smem_bytes(W, max_p1);
    cudaError_t e = raise_smem_limit((const void*)scatter_kernel<W, MAXPER, HI, GATE>, smem);
    if (e != cudaSuccess) return e;
    if (tiles == 0) return cudaSuccess;
    if (tiles > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    scatter_kernel<W, MAXPER, HI, GATE><<<(unsigned)tiles, kStageThreads, smem, s>>>(jobs, tile_off, n_jobs);
    return cudaGetLastError();
}

template <int W, unsigned MAXPER, bool HI>
static cudaError_t launch_scatter_wp(const Job* jobs, const unsigned long long* tile_off, unsigned n_jobs,
                                     unsigned long long tiles, unsigned max_p1, bool gated, cudaStream_t s) {
    return gated ? launch_scatter_wpg<W, MAXPER, HI, true>(jobs, tile_off, n_jobs, tiles, max_p1, s)
                 : launch_scatter_wpg<W, MAXPER, HI, false>(jobs, tile_off, n_jobs, tiles, max_p1, s);
}

template <int W, bool HI>
static cudaError_t launch_scatter_w(const Job* jobs, const unsigned long long* tile_off, unsigned n_jobs,
                                    unsigned long long tiles, unsigned max_p1, bool gated, cudaStream_t s) {
    // MAXPER: destinations of one thread in a flush (fan-out / 256, rounded up to 2, 4 or 8)
    if ((1u << max_p1) <= 2 * kStageThreads)
        return launch_scatter_wp<W, 2, HI>(jobs, tile_off, n_jobs, tiles, max_p1, gated, s);
    if ((1u << max_p1) <= 4 * kStageThreads)
        return launch_scatter_wp<W, 4, HI>(jobs, tile_off, n_jobs, tiles, max_p1, gated, s);
    return launch_scatter_wp<W, kMaxStageDest / kStageThreads, HI>(jobs, tile_off, n_jobs, tiles, max_p1, gated, s);
}

cudaError_t launch_scatter(unsigned W, const Job* jobs, const unsigned long long* tile_off, unsigned n_jobs,
                           unsigned long long tiles, unsigned max_p1, unsigned min_k, bool gated, cudaStream_t s) {
    switch (W) {
        case 1:
            return min_k >= 17 ? launch_scatter_w<1, true>(jobs, tile_off, n_jobs, tiles, max_p1, gated, s)
                               : launch_scatter_w<1, false>(jobs, tile_off, n_jobs, tiles, max_p1, gated, s);
        case 2: return launch_scatter_w<2, false>(jobs, tile_off, n_jobs, tiles, max_p1, gated, s);
        case 3: return launch_scatter_w<3, false>(jobs, tile_off, n_jobs, tiles, max_p1, gated, s);
        case 4: return launch_scatter_w<4, false>(jobs, tile_off, n_jobs, tiles, max_p1, gated, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kmer
