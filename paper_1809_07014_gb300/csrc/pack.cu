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
// number of k-windows for any k; a flag if offsets decrease.  The lanes of a
// warp that share a length bin add to it with one atomic (reads of one run
// usually have the same length).
__global__ void __launch_bounds__(256) read_geometry_kernel(const unsigned long long* offsets, unsigned long long n,
                                                            unsigned long long* nblk, unsigned long long* len_stats,
                                                            unsigned int* bad) {
    __shared__ unsigned long long hist[kLenHist];
    for (int i = threadIdx.x; i < kLenHist; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = blockIdx.x * (unsigned long long)blockDim.x; base < n; base += stride) {
        const unsigned long long r = base + threadIdx.x;
        unsigned bin = 0xFFFFFFFFu;
        unsigned long long L = 0;
        if (r < n) {
            const unsigned long long a = offsets[r], b = offsets[r + 1];
            if (b < a) {
                atomicOr(bad, 1u);
                nblk[r] = 0;
            } else {
                L = b - a;
                nblk[r] = (L + 31) / 32;
                bin = L < kLenExact ? (unsigned)L : (unsigned)kLenExact;
                if (L >= 0x80000000ull) atomicOr(bad, 2u);
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        const bool leader = lane == __ffs(peers) - 1;
        if (bin != 0xFFFFFFFFu && leader) atomicAdd(&hist[bin], (unsigned long long)__popc(peers));
        // lengths of the long reads of this warp, summed over the warp
        unsigned long long ls = bin == (unsigned)kLenExact ? L : 0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
        if (lane == 0 && ls) atomicAdd(&hist[kLenExact + 1], ls);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kLenHist; i += blockDim.x)
        if (hist[i]) atomicAdd(&len_stats[i], hist[i]);
}

// 16 bytes at the 16-byte aligned address c; bytes outside [lo, hi) read as 0.
__device__ __forceinline__ uint4 load16(unsigned long long c, unsigned long long lo, unsigned long long hi) {
    if (c >= lo && c + 16 <= hi) return __ldcs(reinterpret_cast<const uint4*>(c));
    unsigned w[4] = {0u, 0u, 0u, 0u};
#pragma unroll 1
    for (int i = 0; i < 16; ++i) {
        const unsigned long long a = c + i;
        if (a >= lo && a < hi) w[i >> 2] |= (unsigned)*reinterpret_cast<const unsigned char*>(a) << (8 * (i & 3));
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// The 32 bytes starting at address s (any alignment), from three aligned
// 16-byte loads; bytes outside [lo, hi) read as 0.
__device__ __forceinline__ void load32(unsigned long long s, unsigned long long lo, unsigned long long hi,
                                       unsigned (&out)[8]) {
    const unsigned long long c = s & ~15ull;
    const uint4 x0 = load16(c, lo, hi), x1 = load16(c + 16, lo, hi);
    const uint4 x2 = (s & 15ull) ? load16(c + 32, lo, hi) : make_uint4(0u, 0u, 0u, 0u);
    const unsigned w[12] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x2.x, x2.y, x2.z, x2.w};
    const unsigned q = (unsigned)(s & 15ull) >> 2, sh = 8u * (unsigned)(s & 3ull);
    unsigned x[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = q == 0 ? w[i] : (q == 1 ? w[i + 1] : (q == 2 ? w[i + 2] : w[i + 3]));
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = __funnelshift_r(x[i], x[i + 1], sh);
}

// Four bits from the low bit of each byte of v (byte 0 -> bit 0).
__device__ __forceinline__ unsigned byte_lsbs(unsigned v) { return ((v & 0x01010101u) * 0x10204080u) >> 28; }

// One thread per 32-base block.  A warp takes 32 consecutive reads and walks
// their blocks 32 at a time; each lane finds its read by a binary search
// over the lanes' block offsets.  Bases and qualities are read with aligned
// 16-byte loads and classified four bytes at a time.
__global__ void __launch_bounds__(256) pack_kernel(const char* __restrict__ bases, const unsigned char* __restrict__ quals,
                                                  const unsigned long long* __restrict__ offsets,
                                                  const unsigned long long* __restrict__ blk_off, unsigned long long n,
                                                  unsigned hq_min, PackedBlock* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const unsigned long long first_base = offsets[0], end_base = offsets[n];
    const unsigned long long A = reinterpret_cast<unsigned long long>(bases);
    const unsigned long long Q = reinterpret_cast<unsigned long long>(quals);
    const bool hq_never = hq_min > 255u;
    const unsigned thr4 = hq_never ? 0u : hq_min * 0x01010101u;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long r0 = (blockIdx.x * (unsigned long long)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
         r0 < n; r0 += warps * 32) {
        const unsigned nr = (unsigned)(n - r0 < 32 ? n - r0 : 32);
        const unsigned long long r = r0 + lane;
        const bool have = (unsigned)lane < nr;
        const unsigned long long a = have ? offsets[r] : 0ull;
        const unsigned long long L = have ? offsets[r + 1] - a : 0ull;
        const unsigned long long bo = have ? blk_off[r] : ~0ull;
        const unsigned long long first = __shfl_sync(0xffffffffu, bo, 0);
        const unsigned long long last = blk_off[r0 + nr];
        for (unsigned long long B0 = first; B0 < last; B0 += 32) {
            const unsigned long long B = B0 + lane;
            unsigned j = 0;  // the last read whose first block is <= B
#pragma unroll
            for (unsigned st = 16; st; st >>= 1) {
                const unsigned c = j + st;
                const unsigned long long v = __shfl_sync(0xffffffffu, bo, c & 31u);
                if (c < nr && v <= B) j = c;
            }
            const unsigned long long aj = __shfl_sync(0xffffffffu, a, j);
            const unsigned long long Lj = __shfl_sync(0xffffffffu, L, j);
            const unsigned long long bj = __shfl_sync(0xffffffffu, bo, j);
            if (B >= last) continue;
            const unsigned long long pos = 32 * (B - bj);
            const unsigned len = (unsigned)(Lj - pos < 32 ? Lj - pos : 32);
            unsigned cb[8], cq[8];
            load32(A + aj + pos, A + first_base, A + end_base, cb);
            load32(Q + aj + pos, Q + first_base, Q + end_base, cq);
            unsigned long long codes = 0;  // base j at bits 2j, 2j+1 (reversed below)
            unsigned valid = 0, hq = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const unsigned v = cb[i];
                // A, C, G, T (0x41, 0x43, 0x47, 0x54) -> 0, 1, 2, 3: bit 1 ^ bit 2, bit 2 ^ bit 3
                unsigned c2 = ((v >> 1) ^ (v >> 2)) & 0x03030303u;
                // a byte is a base iff it equals the letter of its code: one byte
                // permutation looks up the four letters, an exact zero-byte test compares
                const unsigned x = c2 | (c2 >> 4);
                const unsigned letters = __byte_perm(0x54474341u, 0u, (x & 0xFFu) | ((x >> 8) & 0xFF00u));
                const unsigned t = v ^ letters;
                const unsigned ok = ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t | 0x7F7F7F7Fu);  // 0x80 per base byte
                const unsigned eq = (ok >> 7) * 0xFFu;  // 0xFF per base byte
                c2 &= eq;
                codes |= (unsigned long long)((c2 * 0x01041040u) >> 24) << (8 * i);
                valid |= byte_lsbs(ok >> 7) << (4 * i);
                hq |= byte_lsbs(__vcmpgeu4(cq[i], thr4) & eq) << (4 * i);
            }
            if (hq_never) hq = 0u;
            const unsigned lm = len >= 32 ? 0xFFFFFFFFu : ((1u << len) - 1u);
            valid &= lm;
            hq &= valid;
            codes &= len >= 32 ? ~0ull : ((1ull << (2 * len)) - 1ull);
            // MSB-first: reverse the order of the 2-bit codes
            unsigned long long m = __brevll(codes);
            m = ((m >> 1) & 0x5555555555555555ull) | ((m & 0x5555555555555555ull) << 1);
            PackedBlock pb;
            pb.bases = m;
            pb.nmask = ~valid;
            pb.hqmask = hq;
            out[B] = pb;
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
    const unsigned long long warps = (n + 31) / 32;
    unsigned long long grid = (warps + 7) / 8;
    const unsigned long long cap = (unsigned long long)num_sms * 16;
    if (grid > cap) grid = cap;
    // high quality: Phred + offset >= offset + threshold (never, past a byte)
    const unsigned hq_min = qual_offset + qual_threshold;
    pack_kernel<<<(unsigned)grid, 256, 0, s>>>(bases, quals, offsets, blk_off, n, hq_min, out);
    return cudaGetLastError();
}

}  // namespace kmer
