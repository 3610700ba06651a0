// Step a1: reads (ASCII bases, Phred+offset qualities, base offsets) ->
// packed 2-bit blocks with N and high-quality bit masks.  Reads are strings
// over A, C, G, T (Sec. II, terminology); every other byte is treated as N.
#include "kernels.h"

namespace kmer {

// ---------------------------------------------------------------------------
// Exclusive prefix sum over u64 (three phases: tile sums, scan of the tile
// sums by one CTA, tile scans).  out may alias nothing; out[n] = total.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long* total) {
    __shared__ unsigned long long warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long s = lane < kScanThreads / 32 ? warp_sums[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    unsigned long long before = wid ? warp_sums[wid - 1] : 0ull;
    if (total) *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_sums(const unsigned long long* in, unsigned long long n,
                                                               unsigned long long* tile_sums) {
    const unsigned long long base = (unsigned long long)blockIdx.x * kScanTile;
    unsigned long long s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
        if (base + i < n) s += in[base + i];
    unsigned long long tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_of_sums(unsigned long long* sums, unsigned long long n_tiles) {
    unsigned long long carry = 0;
    for (unsigned long long b = 0; b < n_tiles; b += kScanThreads) {
        unsigned long long i = b + threadIdx.x;
        unsigned long long v = i < n_tiles ? sums[i] : 0ull, tot;
        unsigned long long ex = block_exclusive_scan(v, &tot);
        if (i < n_tiles) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[n_tiles] = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles(const unsigned long long* in, unsigned long long n,
                                                           const unsigned long long* tile_prefix,
                                                           unsigned long long* out) {
    const unsigned long long base = (unsigned long long)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    unsigned long long v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0ull;
        s += v[i];
    }
    unsigned long long run = block_exclusive_scan(s, nullptr) + tile_prefix[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = tile_prefix[gridDim.x];
}

size_t scan_temp_bytes(unsigned long long n) { return ((n + kScanTile - 1) / kScanTile + 1) * 8 + 256; }

cudaError_t exclusive_scan_u64(const unsigned long long* in, unsigned long long* out, unsigned long long n,
                               void* temp, cudaStream_t s) {
    unsigned long long tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) tiles = 1;
    auto* sums = static_cast<unsigned long long*>(temp);
    scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
    scan_of_sums<<<1, kScanThreads, 0, s>>>(sums, tiles);
    scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per read: number of 32-base blocks; a histogram of read lengths (< 128
// exactly, >= 128 as count and sum) from which the host computes the exact
// number of k-windows for any k; a flag if offsets decrease.
__global__ void read_geometry_kernel(const unsigned long long* offsets, unsigned long long n,
                                     unsigned long long* nblk, unsigned long long* len_stats,
                                     unsigned int* bad) {
    __shared__ unsigned long long hist[kLenHist];
    for (int i = threadIdx.x; i < kLenHist; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < n;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long a = offsets[r], b = offsets[r + 1];
        if (b < a) {
            atomicOr(bad, 1u);
            nblk[r] = 0;
            continue;
        }
        unsigned long long L = b - a;
        nblk[r] = (L + 31) / 32;
        if (L < kLenExact) {
            atomicAdd(&hist[L], 1ull);
        } else {
            atomicAdd(&hist[kLenExact], 1ull);
            atomicAdd(&hist[kLenExact + 1], L);
        }
        if (L >= 0x80000000ull) atomicOr(bad, 2u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kLenHist; i += blockDim.x)
        if (hist[i]) atomicAdd(&len_stats[i], hist[i]);
}

// One warp per read: lane j handles base 32*blk + j of the read, so each load
// instruction reads 32 consecutive bytes.  The 2-bit codes are gathered with
// two warp OR-reductions (bases 0..15 -> high half, 16..31 -> low half).
__global__ void __launch_bounds__(256) pack_kernel(const char* __restrict__ bases, const unsigned char* __restrict__ quals,
                                                  const unsigned long long* __restrict__ offsets,
                                                  const unsigned long long* __restrict__ blk_off, unsigned long long n,
                                                  unsigned qual_offset, unsigned qual_threshold,
                                                  PackedBlock* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long r = blockIdx.x * (unsigned long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < n;
         r += warps) {
        const unsigned long long a = offsets[r], L = offsets[r + 1] - a, ob = blk_off[r];
        const unsigned long long nb = (L + 31) / 32;
        for (unsigned long long blk = 0; blk < nb; ++blk) {
            const unsigned long long pos = blk * 32 + lane;
            unsigned code = 0, isn = 1, hq = 0;
            if (pos < L) {
                const unsigned char c = (unsigned char)bases[a + pos];
                const unsigned q = quals[a + pos];
                switch (c) {
                    case 'A': code = 0; isn = 0; break;
                    case 'C': code = 1; isn = 0; break;
                    case 'G': code = 2; isn = 0; break;
                    case 'T': code = 3; isn = 0; break;
                    default: break;
                }
                hq = (q >= qual_offset && q - qual_offset >= qual_threshold) ? 1u : 0u;
            }
            const unsigned hi_part = lane < 16 ? code << (30 - 2 * lane) : 0u;
            const unsigned lo_part = lane >= 16 ? code << (30 - 2 * (lane - 16)) : 0u;
            const unsigned hi = __reduce_or_sync(0xffffffffu, hi_part);
            const unsigned lo = __reduce_or_sync(0xffffffffu, lo_part);
            const unsigned nm = __ballot_sync(0xffffffffu, isn != 0);
            const unsigned hm = __ballot_sync(0xffffffffu, hq != 0 && isn == 0);
            if (lane == 0) {
                PackedBlock pb;
                pb.bases = ((unsigned long long)hi << 32) | lo;
                pb.nmask = nm;
                pb.hqmask = hm;
                out[ob + blk] = pb;
            }
        }
    }
}

cudaError_t launch_read_geometry(const unsigned long long* offsets, unsigned long long n, unsigned long long* nblk,
                                 unsigned long long* len_stats, unsigned int* bad, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unsigned long long grid = (n + 255) / 256;
    if (grid > 4096) grid = 4096;
    read_geometry_kernel<<<(unsigned)grid, 256, 0, s>>>(offsets, n, nblk, len_stats, bad);
    return cudaGetLastError();
}

cudaError_t launch_pack(const char* bases, const unsigned char* quals, const unsigned long long* offsets,
                        const unsigned long long* blk_off, unsigned long long n, unsigned qual_offset,
                        unsigned qual_threshold, PackedBlock* out, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unsigned long long grid = (n + 7) / 8;
    const unsigned long long cap = (unsigned long long)num_sms * 8 * 4;
    if (grid > cap) grid = cap;
    pack_kernel<<<(unsigned)grid, 256, 0, s>>>(bases, quals, offsets, blk_off, n, qual_offset, qual_threshold, out);
    return cudaGetLastError();
}

}  // namespace kmer
