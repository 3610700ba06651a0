// Survivors in ascending key order (KMER_FLAG_SORTED_OUTPUT).  The k-mer set
// is a set (Sec. II-A use case 1: inserts commute), so its order is free; the
// partitions leave it grouped by the mixed key.  A least-significant-digit
// radix sort of the keys (8-bit digits over the 2k key bits) carries each
// survivor's position along; the counts, tallies and classes travel as one
// 64-byte record per survivor (written while the digits are counted) and are
// gathered through that permutation straight into the result arrays, one
// random record read per survivor (three random reads of the separate arrays
// and a copy back took about 30 % longer on 114 M survivors).
//
// One kernel per digit (a one-sweep pass): each CTA takes the next tile of
// keys, ranks them by digit within the tile (stable: warps own consecutive
// runs of keys, lanes of one digit are ordered by lane), publishes its
// per-digit counts, and sums the counts of the tiles before it by looking
// back along a per-(tile, digit) status array (decoupled look-back: a tile's
// inclusive prefix, once known, ends the walk of every later tile).  The
// tile is then reordered by digit in shared memory and written out, so each
// digit's keys leave as one contiguous run.  The digit totals of every pass
// come from one histogram kernel over the keys; passes whose digit is the
// same for every key are skipped.
#include <vector>

#include "kernels.h"

namespace kmer {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr unsigned kSortSpinBudget = 1u << 22;  // look-back polls per thread before giving up
constexpr int kLookBack = 8;                     // predecessors read per look-back step

template <int W>
struct SortShape {
    // keys per thread and CTAs per SM (the registers are bounded for it): a
    // pass holds only one word per key in registers, so occupancy is set by
    // the shared-memory tile; measured on 114 M one-word keys, 8 keys at six
    // CTAs per SM ran a pass in 0.86 ms against 1.16 ms for 12 keys at three
    static constexpr int ITEMS = W <= 2 ? 8 : 4;
    static constexpr int MINB = W == 1 ? 6 : 4;
    static constexpr int TILE = kSortThreads * ITEMS;
    static constexpr size_t SMEM = (size_t)TILE * W * 8 + (size_t)TILE * 4;  // reordered keys + positions
};

// Digit `pass` (bits [8 pass, 8 pass + 8) of the key value) of a key: word
// W - 1 - 8 pass / 64, shifted right by 8 pass % 64 (a select, not an indexed
// load, so the key stays in registers).
template <int W>
__device__ __forceinline__ unsigned digit_of(const unsigned long long (&key)[W], unsigned pass) {
    const unsigned wi = W - 1 - (8 * pass) / 64, sh = (8 * pass) % 64;
    unsigned long long v = key[0];
#pragma unroll
    for (int w = 1; w < W; ++w) v = (unsigned)w == wi ? key[w] : v;
    return (unsigned)(v >> sh) & 0xFFu;
}

// A survivor's payload while the keys are sorted, 64 bytes (written whole,
// so no sector is partly written): (count, classes left | right << 8, 0, 0),
// ext[0..3], ext[4..7], zeros.
constexpr int kRecU4 = 4;

// hist[p * 256 + d] = keys whose digit p is d, for p < passes; rec[i] = the
// payload record of survivor i.
template <int W>
__global__ void __launch_bounds__(kSortThreads) sort_digits_kernel(const unsigned long long* __restrict__ keys,
                                                                   const unsigned* __restrict__ count,
                                                                   const unsigned* __restrict__ ext,
                                                                   const unsigned char* __restrict__ cls,
                                                                   unsigned long long n, unsigned passes,
                                                                   unsigned* __restrict__ hist,
                                                                   uint4* __restrict__ rec) {
    extern __shared__ unsigned h[];  // passes * 256
    for (unsigned i = threadIdx.x; i < passes * 256; i += kSortThreads) h[i] = 0;
    __syncthreads();
    for (unsigned long long i = blockIdx.x * (unsigned long long)kSortThreads + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * kSortThreads) {
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = keys[i * W + w];
        const uchar2 c2 = reinterpret_cast<const uchar2*>(cls)[i];
        const uint4* e = reinterpret_cast<const uint4*>(ext + i * 8);
        uint4* r = rec + i * kRecU4;
        r[0] = make_uint4(count[i], (unsigned)c2.x | (unsigned)c2.y << 8, 0u, 0u);
        r[1] = e[0];
        r[2] = e[1];
        r[3] = make_uint4(0u, 0u, 0u, 0u);
        for (unsigned p = 0; p < passes; ++p) atomicAdd(&h[p * 256 + digit_of<W>(key, p)], 1u);
    }
    __syncthreads();
    for (unsigned i = threadIdx.x; i < passes * 256; i += kSortThreads)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

__device__ __forceinline__ unsigned long long poll(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void publish(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive scan of one value per thread over the CTA (256 threads).
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* warp_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    unsigned before = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w)
        if (w < wid) before += warp_tot[w];
    __syncthreads();
    return before + x - v;
}

// One pass: keys (and positions; identity when isrc is null) from src to dst
// ordered by digit `pass`.  status: tiles * 256 words (stamp << 32 | count),
// stamps 2 s + 1 (the tile's own count) and 2 s + 2 (its inclusive prefix)
// for the s-th pass of this sort; tile_counter: zero before the pass.
// Only the key word that holds the digit is kept in registers while ranking;
// the keys and positions are read again (from L2) when the tile is reordered,
// and the look-back runs after the reorder so its wait overlaps that work.
template <int W>
__global__ void __launch_bounds__(kSortThreads, SortShape<W>::MINB) sort_pass_kernel(
    const unsigned long long* __restrict__ src, const unsigned* __restrict__ isrc, unsigned long long n,
    unsigned pass, unsigned stamp_s, const unsigned* __restrict__ hist, unsigned long long* status,
    unsigned* tile_counter, unsigned long long* __restrict__ dst, unsigned* __restrict__ idst, unsigned* err) {
    constexpr int ITEMS = SortShape<W>::ITEMS, TILE = SortShape<W>::TILE;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* skeys = reinterpret_cast<unsigned long long*>(smem);
    unsigned* sidx = reinterpret_cast<unsigned*>(smem + (size_t)TILE * W * 8);
    __shared__ unsigned wcnt[kSortWarps][256];  // per warp: keys per digit, then its first rank in the tile
    __shared__ unsigned tstart[256];            // tile-local start of each digit
    __shared__ unsigned long long gbase[256];   // global start of the tile's run of each digit
    __shared__ unsigned warp_tot[kSortWarps];
    __shared__ unsigned s_tile;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned d_me = threadIdx.x;  // the digit this thread looks after in the scans
    const unsigned wi = W - 1 - (8 * pass) / 64, sh = (8 * pass) % 64;  // the digit's word and shift
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);  // tiles in start order: predecessors run
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const unsigned long long t = s_tile;
    const unsigned long long t0 = t * TILE;
    const unsigned tile_n = (unsigned)(n - t0 < (unsigned long long)TILE ? n - t0 : TILE);

    // ---- digits and ranks: warp w owns keys [w * 32 * ITEMS, (w + 1) * 32 * ITEMS) of the tile
    unsigned dr[ITEMS];  // digit (9 bits: 256 + lane past the end), then rank << 9 | digit
    const unsigned long long wbase = t0 + (unsigned long long)wid * 32 * ITEMS;
#pragma unroll
    for (int u = 0; u < ITEMS; ++u) {
        const unsigned long long i = wbase + (unsigned long long)u * 32 + lane;
        dr[u] = i < n ? (unsigned)(src[i * W + wi] >> sh) & 0xFFu : 256u + lane;  // past the end: a digit of its own
    }
#pragma unroll
    for (int u = 0; u < ITEMS; ++u) {
        const unsigned d = dr[u];
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned before = __popc(peers & ((1u << lane) - 1u));
        const bool in = d < 256;
        const unsigned run = in ? wcnt[wid][d] : 0u;
        __syncwarp();
        if (in && before == 0) wcnt[wid][d] = run + __popc(peers);
        __syncwarp();
        dr[u] = (run + before) << 9 | d;  // rank among the warp's keys of digit d
    }
    __syncthreads();

    // ---- tile counts per digit: publish them; tile-local starts
    unsigned cnt = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const unsigned c = wcnt[w][d_me];
        wcnt[w][d_me] = cnt;  // warps' first ranks within the digit
        cnt += c;
    }
    const unsigned agg = 2 * stamp_s + 1, inc = 2 * stamp_s + 2;
    unsigned long long* my = status + t * 256 + d_me;
    publish(my, (unsigned long long)(t == 0 ? inc : agg) << 32 | cnt);
    // start of the digit's run among all keys: earlier digits of this pass
    const unsigned dstart = block_excl_scan(__ldg(hist + pass * 256 + d_me), warp_tot);
    tstart[d_me] = block_excl_scan(cnt, warp_tot);
    __syncthreads();

    // ---- reorder the tile by digit in shared memory (keys and positions read again)
#pragma unroll
    for (int u = 0; u < ITEMS; ++u) {
        const unsigned d = dr[u] & 0x1FFu;
        if (d >= 256) continue;
        const unsigned long long i = wbase + (unsigned long long)u * 32 + lane;
        const unsigned lp = tstart[d] + wcnt[wid][d] + (dr[u] >> 9);
#pragma unroll
        for (int w = 0; w < W; ++w) skeys[(size_t)lp * W + w] = src[i * W + w];
        sidx[lp] = isrc ? isrc[i] : (unsigned)i;
    }

    // ---- look-back: keys of this digit in earlier tiles
    unsigned long long prefix = 0;
    if (t > 0) {
        // a window of kLookBack predecessors per step: their words are read
        // together and summed nearest first up to the first inclusive prefix;
        // a predecessor that has not yet published is polled again
        unsigned spins = 0;
        bool gave_up = false;
        long long j = (long long)t - 1;
        for (;;) {
            unsigned long long v[kLookBack];
#pragma unroll
            for (int q = 0; q < kLookBack; ++q)
                v[q] = j - q >= 0 ? poll(status + (unsigned long long)(j - q) * 256 + d_me)
                                  : (unsigned long long)inc << 32;  // before tile 0: an empty prefix
            int q = 0;
            bool done = false;
            for (; q < kLookBack; ++q) {
                const unsigned st = (unsigned)(v[q] >> 32);
                if (st != agg && st != inc) break;
                prefix += v[q] & 0xFFFFFFFFull;
                if (st == inc) {
                    done = true;
                    break;
                }
            }
            if (done) break;
            j -= q;
            if (q < kLookBack) {
                if (++spins > kSortSpinBudget) {
                    gave_up = true;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (gave_up) atomicOr(err, ST_TIMEOUT);
        publish(my, (unsigned long long)inc << 32 | ((prefix + cnt) & 0xFFFFFFFFull));
    }
    gbase[d_me] = (unsigned long long)dstart + prefix;
    __syncthreads();

    // ---- write each digit's run
    for (unsigned j = threadIdx.x; j < tile_n; j += kSortThreads) {
        const unsigned d = (unsigned)(skeys[(size_t)j * W + wi] >> sh) & 0xFFu;
        const unsigned long long g = gbase[d] + (j - tstart[d]);
        if (g >= n) {  // only after a look-back gave up: record it and skip the write
            atomicOr(err, ST_SORT_RANGE);
            continue;
        }
#pragma unroll
        for (int w = 0; w < W; ++w) dst[g * W + w] = skeys[(size_t)j * W + w];
        idst[g] = sidx[j];
    }
}

// The survivors' counts, tallies and classes in the order of `perm`, from
// their payload records (`ext` 16-byte and `cls` 2-byte aligned, as the
// result arrays always are).
__global__ void __launch_bounds__(256) sort_gather_kernel(const unsigned* __restrict__ perm, unsigned long long n,
                                                          const uint4* __restrict__ rec,
                                                          unsigned* __restrict__ count, unsigned* __restrict__ ext,
                                                          unsigned char* __restrict__ cls) {
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * 256) {
        const uint4* r = rec + (unsigned long long)perm[i] * kRecU4;
        const uint4 a = r[0], e0 = r[1], e1 = r[2];
        count[i] = a.x;
        uint4* eo = reinterpret_cast<uint4*>(ext + i * 8);
        eo[0] = e0;
        eo[1] = e1;
        reinterpret_cast<uchar2*>(cls)[i] = make_uchar2((unsigned char)(a.y & 0xFFu), (unsigned char)(a.y >> 8));
    }
}

static size_t carved(size_t b) { return (b + 255) & ~size_t(255); }

static unsigned sort_passes(unsigned k) { return (2 * k + 7) / 8; }

static unsigned long long sort_tiles(unsigned W, unsigned long long n) {
    const unsigned long long T = W == 1   ? SortShape<1>::TILE
                                 : W == 2 ? SortShape<2>::TILE
                                 : W == 3 ? SortShape<3>::TILE
                                          : SortShape<4>::TILE;
    return (n + T - 1) / T;
}

size_t sort_scratch_bytes(unsigned W, unsigned long long n) {
    const unsigned passes = sort_passes(32 * W);  // enough for any k of this width
    return carved(n * 8 * W) + 2 * carved(n * 4) + carved(sort_tiles(W, n) * 256 * 8) + carved(passes * 256 * 4) +
           carved(passes * 4) + carved(n * 16 * kRecU4);
}

template <int W>
static cudaError_t sort_w(unsigned long long* keys, unsigned* count, unsigned* ext, unsigned char* cls,
                          unsigned long long n, unsigned k, void* scratch, unsigned* status, int num_sms,
                          unsigned* launches, cudaStream_t s) {
    using Shape = SortShape<W>;
    const unsigned long long tiles = (n + Shape::TILE - 1) / Shape::TILE;
    const unsigned passes = sort_passes(k);
    unsigned char* p = static_cast<unsigned char*>(scratch);
    auto carve = [&](size_t bytes) {
        unsigned char* r = p;
        p += carved(bytes);
        return r;
    };
    unsigned long long* kb = reinterpret_cast<unsigned long long*>(carve(n * 8 * W));
    unsigned* ia = reinterpret_cast<unsigned*>(carve(n * 4));
    unsigned* ib = reinterpret_cast<unsigned*>(carve(n * 4));
    unsigned long long* st = reinterpret_cast<unsigned long long*>(carve(tiles * 256 * 8));
    unsigned* hist = reinterpret_cast<unsigned*>(carve(passes * 256 * 4));
    unsigned* counters = reinterpret_cast<unsigned*>(carve(passes * 4));
    uint4* rec = reinterpret_cast<uint4*>(carve(n * 16 * kRecU4));
    cudaError_t e = cudaMemsetAsync(st, 0, tiles * 256 * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, passes * 256 * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, passes * 4, s);
    if (e != cudaSuccess) return e;
    // digit totals of every pass (passes whose digit is the same for every key
    // move nothing) and the payload records
    const size_t hsmem = passes * 256 * 4;
    e = raise_smem_limit((const void*)sort_digits_kernel<W>, hsmem);
    if (e != cudaSuccess) return e;
    const unsigned long long hb = (n + kSortThreads - 1) / kSortThreads;
    const unsigned hgrid = (unsigned)(hb < (unsigned long long)num_sms * 16 ? hb : num_sms * 16);
    sort_digits_kernel<W><<<hgrid, kSortThreads, hsmem, s>>>(keys, count, ext, cls, n, passes, hist, rec);
    ++*launches;
    std::vector<unsigned> h(passes * 256);
    e = cudaMemcpyAsync(h.data(), hist, h.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    e = raise_smem_limit((const void*)sort_pass_kernel<W>, Shape::SMEM);
    if (e != cudaSuccess) return e;
    // keys move from `keys` to the scratch and back, pass by pass (a final
    // copy into `keys` when the number of passes that moved is odd)
    const unsigned long long* src = keys;
    const unsigned* isrc = nullptr;
    unsigned long long* bufs[2] = {kb, keys};
    unsigned* ibufs[2] = {ia, ib};
    unsigned moved = 0;
    for (unsigned pass = 0; pass < passes; ++pass) {
        unsigned nz = 0;
        for (int d = 0; d < 256; ++d) nz += h[pass * 256 + d] != 0;
        if (nz <= 1) continue;
        unsigned long long* dst = bufs[moved & 1];
        unsigned* idst = ibufs[moved & 1];
        sort_pass_kernel<W><<<(unsigned)tiles, kSortThreads, Shape::SMEM, s>>>(
            src, isrc, n, pass, moved, hist, st, counters + pass, dst, idst, status);
        ++*launches;
        src = dst;
        isrc = idst;
        ++moved;
    }
    if (!moved) return cudaGetLastError();  // a single key value: nothing moves
    if (src != keys) {
        e = cudaMemcpyAsync(keys, src, n * 8 * W, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    const unsigned long long gb = (n + 255) / 256;
    const unsigned g = (unsigned)(gb < (unsigned long long)num_sms * 32 ? gb : num_sms * 32);
    sort_gather_kernel<<<g, 256, 0, s>>>(isrc, n, rec, count, ext, cls);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_sort_survivors(unsigned W, unsigned long long* keys, unsigned* count, unsigned* ext,
                                  unsigned char* cls, unsigned long long n, unsigned k, void* scratch,
                                  unsigned* status, int num_sms, unsigned* launches, cudaStream_t s) {
    if (n < 2) return cudaSuccess;
    if (n >= 0xFFFFFFFFull || (2 * k + 63) / 64 != W) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(keys) & 7) || (reinterpret_cast<uintptr_t>(count) & 3) ||
        (reinterpret_cast<uintptr_t>(ext) & 15) || (reinterpret_cast<uintptr_t>(cls) & 1))
        return cudaErrorInvalidValue;
    switch (W) {
        case 1: return sort_w<1>(keys, count, ext, cls, n, k, scratch, status, num_sms, launches, s);
        case 2: return sort_w<2>(keys, count, ext, cls, n, k, scratch, status, num_sms, launches, s);
        case 3: return sort_w<3>(keys, count, ext, cls, n, k, scratch, status, num_sms, launches, s);
        case 4: return sort_w<4>(keys, count, ext, cls, n, k, scratch, status, num_sms, launches, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kmer
