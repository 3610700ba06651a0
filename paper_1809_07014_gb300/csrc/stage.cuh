// Shared-memory staging of partitioned records: records of one round are
// counted per destination in shared memory, one global atomic per
// destination reserves their slots, and the records are written out sorted
// by destination so that each warp stores contiguous runs.  This is the
// aggregation of fine-grained inserts into batch updates that the paper
// describes for update-only hash-table phases (Sec. II-A, use case 1).
#pragma once
#include "common.cuh"

namespace kmer {

constexpr int kStageThreads = 256;
constexpr unsigned kMaxStageDest = 2048;  // destinations of one staging round (partition fan-out)

// Exclusive scan across the NT threads of the block (all must call;
// warp_tmp holds NT / 32 words).
template <unsigned NT = kStageThreads>
__device__ inline unsigned block_scan_u32(unsigned v, unsigned* warp_tmp, unsigned* total) {
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned s = lane < (int)(NT / 32) ? warp_tmp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < (int)(NT / 32)) warp_tmp[lane] = s;
    }
    __syncthreads();
    const unsigned before = wid ? warp_tmp[wid - 1] : 0u;
    *total = warp_tmp[NT / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// 64-bit variant (warp_tmp must hold 8 u64).
__device__ inline unsigned long long block_scan_u64(unsigned long long v, unsigned long long* warp_tmp,
                                                    unsigned long long* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long s = lane < kStageThreads / 32 ? warp_tmp[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kStageThreads / 32) warp_tmp[lane] = s;
    }
    __syncthreads();
    const unsigned long long before = wid ? warp_tmp[wid - 1] : 0ull;
    *total = warp_tmp[kStageThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

struct StageBufs {
    unsigned long long* stage;   // S * W: records in arrival order
    unsigned long long* wbase;   // P: record index of sorted position 0 of destination d
    unsigned* ok_end;            // P: first sorted position of destination d past its capacity
    unsigned* meta;              // S
    unsigned* hist;              // P
    unsigned* lbase;             // P
    unsigned* order;             // S: (destination << 16) | staged index, per sorted position
    unsigned* warp_tmp;          // one word per warp of the block (up to 32)
};

__host__ __device__ inline size_t stage_smem_bytes(unsigned W, unsigned S, unsigned P) {
    return (size_t)S * W * 8 + (size_t)P * 8 + (size_t)P * 4 + (size_t)S * 4 + (size_t)P * 8 + (size_t)S * 4 + 128;
}

__device__ inline StageBufs carve_stage(unsigned char* base, unsigned W, unsigned S, unsigned P) {
    StageBufs b;
    b.stage = reinterpret_cast<unsigned long long*>(base);
    b.wbase = b.stage + (size_t)S * W;
    b.ok_end = reinterpret_cast<unsigned*>(b.wbase + P);
    b.meta = b.ok_end + P;
    b.hist = b.meta + S;
    b.lbase = b.hist + P;
    b.order = b.lbase + P;
    b.warp_tmp = b.order + S;
    return b;
}

// Flush one round.  meta[e] = (dest << 16) | rank for a staged record e, or
// 0xFFFFFFFF; hist[d] = records staged for destination d (S <= 65536).  Dest
// supplies reserve(d, n) -> first slot index within d, start(d) -> record
// index of slot 0 of d, cap(d) -> slots of d.  Records past cap are dropped
// and reported through `status` (the host then retries with exact
// capacities).  hist is left zeroed for the next round.
//
// The records are not moved inside shared memory: a word per sorted position
// says which staged record goes there and to which destination, and
// consecutive threads write consecutive positions, i.e. contiguous runs per
// destination.
//
// `sort` places every staged record's word in `order` once the local bases
// are known (from meta[] in shared memory, or from registers).
template <int W, unsigned MAXPER, class Dest, unsigned NT, class Sort>
__device__ __forceinline__ void flush_stage_with(const StageBufs& b, unsigned S, unsigned P, Dest& dest,
                                                 unsigned long long* out_rec, unsigned* status,
                                                 unsigned overflow_bit, Sort sort) {
    __syncthreads();
    // exclusive scan of hist -> lbase (each thread owns a run of consecutive destinations)
    const unsigned per = (P + NT - 1) / NT;
    const unsigned d0 = threadIdx.x * per;
    unsigned mine = 0;
    for (unsigned i = 0; i < per; ++i)
        if (d0 + i < P) mine += b.hist[d0 + i];
    unsigned total;
    const unsigned run0 = block_scan_u32<NT>(mine, b.warp_tmp, &total);
    // reservations of this thread's destinations are independent: all are
    // issued together, and their results are only used after the sort below
    // (which needs just the local bases), so the atomics' latency overlaps it
    unsigned long long first[MAXPER];
    unsigned hs[MAXPER];
    unsigned run = run0;
#pragma unroll
    for (unsigned i = 0; i < MAXPER; ++i) {
        const unsigned d = d0 + i;
        hs[i] = 0;
        first[i] = 0;
        if (i < per && d < P) {
            hs[i] = b.hist[d];
            b.lbase[d] = run;
            if (hs[i]) first[i] = dest.reserve(d, hs[i]);
            run += hs[i];
        }
    }
    __syncthreads();
    sort();
    bool over = false;
    run = run0;
#pragma unroll
    for (unsigned i = 0; i < MAXPER; ++i) {
        const unsigned d = d0 + i;
        const unsigned h = hs[i];
        if (h) {
            const unsigned long long cap = dest.cap(d);
            b.wbase[d] = dest.start(d) + first[i] - run;
            // positions of d that still fit: [run, run + min(h, cap - first))
            const unsigned long long room = first[i] < cap ? cap - first[i] : 0ull;
            b.ok_end[d] = run + (unsigned)(room < h ? room : h);
            over = over || room < h;
        }
        run += h;
    }
    __syncthreads();
    for (unsigned pos = threadIdx.x; pos < total; pos += NT) {
        const unsigned o = b.order[pos];
        const unsigned d = o >> 16, e = o & 0xFFFFu;
        if (pos < b.ok_end[d]) {
            const unsigned long long g = b.wbase[d] + pos;
#pragma unroll
            for (int w = 0; w < W; ++w) out_rec[g * W + w] = b.stage[(size_t)e * W + w];
        }
    }
    for (unsigned d = threadIdx.x; d < P; d += NT) b.hist[d] = 0;
    if (over) atomicOr(status, overflow_bit);
    __syncthreads();
}

// Sorted position of staged record e with meta word m (see flush_stage).
__device__ __forceinline__ void place(const StageBufs& b, unsigned m, unsigned e) {
    if (m != 0xFFFFFFFFu) b.order[b.lbase[m >> 16] + (m & 0xFFFFu)] = (m & 0xFFFF0000u) | e;
}

// Meta words in shared memory (meta[e] for every staged record e).
template <int W, unsigned MAXPER, class Dest, unsigned NT = kStageThreads>
__device__ void flush_stage(const StageBufs& b, unsigned S, unsigned P, Dest& dest, unsigned long long* out_rec,
                            unsigned* status, unsigned overflow_bit) {
    flush_stage_with<W, MAXPER, Dest, NT>(b, S, P, dest, out_rec, status, overflow_bit, [&]() {
        for (unsigned e = threadIdx.x; e < S; e += NT) place(b, b.meta[e], e);
    });
}

// Meta words in registers: m[u] belongs to staged record u * NT + threadIdx.x.
template <int W, unsigned MAXPER, class Dest, unsigned NT, unsigned U>
__device__ void flush_stage_regs(const StageBufs& b, unsigned S, unsigned P, Dest& dest, unsigned long long* out_rec,
                                 unsigned* status, unsigned overflow_bit, const unsigned (&m)[U]) {
    flush_stage_with<W, MAXPER, Dest, NT>(b, S, P, dest, out_rec, status, overflow_bit, [&]() {
#pragma unroll
        for (unsigned u = 0; u < U; ++u) place(b, m[u], u * NT + threadIdx.x);
    });
}

}  // namespace kmer
