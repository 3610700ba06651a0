// Point lookups of k-mers among the survivors of a query: the read side of
// the k-mer table that the later stages of Algorithm 1 consult (the de
// Bruijn graph walks of Sec. II-C ask, for a k-mer, its count and the class
// of each side).  An index over the compacted survivors -- an open-addressing
// table of survivor positions in HBM -- is built once per query; each lookup
// canonicalises the given k-mer (Sec. II-B: a k-mer and its reverse
// complement are one vertex) and probes the index.
#include "kernels.h"
#include "keyops.cuh"
#include "kmer_analysis.h"

namespace kmer {

template <int W>
__global__ void __launch_bounds__(256) index_build_kernel(const unsigned long long* __restrict__ keys,
                                                          unsigned long long n, unsigned* __restrict__ idx,
                                                          unsigned long long cap) {
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * 256) {
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = keys[i * W + w];
        unsigned long long s = key_hash<W>(key) & (cap - 1);
        // survivors are distinct keys: the first empty slot of the sequence is ours
        for (unsigned long long probe = 0; probe < cap; ++probe) {
            if (atomicCAS(idx + s, kIdxEmpty, (unsigned)i) == kIdxEmpty) break;
            s = (s + 1) & (cap - 1);
        }
    }
}

template <int W>
__global__ void __launch_bounds__(256) lookup_kernel(const unsigned long long* __restrict__ q, unsigned long long n,
                                                     const unsigned k, const unsigned* __restrict__ idx,
                                                     unsigned long long cap, const unsigned long long* __restrict__ keys,
                                                     const unsigned* __restrict__ count,
                                                     const unsigned* __restrict__ ext,
                                                     const unsigned char* __restrict__ cls,
                                                     kmer_record* __restrict__ out) {
    const unsigned hb = 2 * k - 64 * (W - 1);
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * 256) {
        unsigned long long key[W], rc[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            key[w] = q[i * W + w];
            rc[w] = 0;
        }
        kmer_record r{};
        const bool valid = hb >= 64 || (key[0] >> hb) == 0ull;  // no bits above 2k
        if (valid) {
            for (unsigned b = 0; b < k; ++b) set_base<W>(rc, k, k - 1 - b, 3u - get_base<W>(key, k, b));
            bool flip = false;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (key[w] != rc[w]) {
                    flip = rc[w] < key[w];
                    break;
                }
            }
            if (flip) {
#pragma unroll
                for (int w = 0; w < W; ++w) key[w] = rc[w];
            }
            r.flipped = flip ? 1 : 0;
            unsigned long long s = key_hash<W>(key) & (cap - 1);
            for (unsigned long long probe = 0; probe < cap; ++probe) {
                const unsigned p = idx[s];
                if (p == kIdxEmpty) break;
                bool same = true;
#pragma unroll
                for (int w = 0; w < W; ++w) same = same && keys[(unsigned long long)p * W + w] == key[w];
                if (same) {
                    r.found = 1;
                    r.count = count[p];
#pragma unroll
                    for (int e = 0; e < 8; ++e) r.ext[e] = ext[(unsigned long long)p * 8 + e];
                    r.cls[0] = cls[2ull * p];
                    r.cls[1] = cls[2ull * p + 1];
                    break;
                }
                s = (s + 1) & (cap - 1);
            }
        }
        out[i] = r;
    }
}

// Merge of Algorithm 1 (Sec. II-G): every k-mer of a second set (the
// contigs' k-mers, canonical and distinct) that is not among the survivors
// is appended to the survivors with count 0, zero tallies and its own
// classes; one that is already there keeps the survivor's record (the two
// occurrences collapse into one).  The index covers the survivors present
// before the merge; `n_out` counts appended positions (one reservation per
// warp).
template <int W>
__global__ void __launch_bounds__(256) merge_append_kernel(const unsigned long long* __restrict__ bkeys,
                                                           const unsigned char* __restrict__ bcls,
                                                           unsigned long long bn, const unsigned* __restrict__ idx,
                                                           unsigned long long cap, unsigned long long* keys,
                                                           unsigned* count, unsigned* ext, unsigned char* cls,
                                                           unsigned long long out_cap,
                                                           unsigned long long* __restrict__ n_out,
                                                           unsigned* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * 256;
    for (unsigned long long base = blockIdx.x * 256ull + (threadIdx.x & ~31u); base < bn; base += stride) {
        const unsigned long long i = base + lane;
        bool add = false;
        unsigned long long key[W];
        if (i < bn) {
#pragma unroll
            for (int w = 0; w < W; ++w) key[w] = bkeys[i * W + w];
            add = true;
            unsigned long long s = key_hash<W>(key) & (cap - 1);
            for (unsigned long long probe = 0; probe < cap; ++probe) {
                const unsigned p = idx[s];
                if (p == kIdxEmpty) break;
                bool same = true;
#pragma unroll
                for (int w = 0; w < W; ++w) same = same && keys[(unsigned long long)p * W + w] == key[w];
                if (same) {
                    add = false;
                    break;
                }
                s = (s + 1) & (cap - 1);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, add);
        unsigned long long first = 0;
        if (lane == 0 && m) first = atomicAdd(n_out, (unsigned long long)__popc(m));
        first = __shfl_sync(0xffffffffu, first, 0);
        if (add) {
            const unsigned long long pos = first + __popc(m & ((1u << lane) - 1u));
            if (pos >= out_cap) {
                atomicOr(status, 1u);
            } else {
#pragma unroll
                for (int w = 0; w < W; ++w) keys[pos * W + w] = key[w];
                count[pos] = 0;
                uint4* eo = reinterpret_cast<uint4*>(ext + pos * 8);
                eo[0] = make_uint4(0, 0, 0, 0);
                eo[1] = make_uint4(0, 0, 0, 0);
                cls[2 * pos] = bcls[2 * i];
                cls[2 * pos + 1] = bcls[2 * i + 1];
            }
        }
    }
}

static unsigned grid_of(unsigned long long n, int num_sms) {
    unsigned long long g = (n + 255) / 256, cap = (unsigned long long)num_sms * 8;
    if (g > cap) g = cap;
    return g ? (unsigned)g : 1u;
}

cudaError_t launch_index_build(unsigned W, const unsigned long long* keys, unsigned long long n, unsigned* idx,
                               unsigned long long cap, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned g = grid_of(n, num_sms);
    switch (W) {
        case 1: index_build_kernel<1><<<g, 256, 0, s>>>(keys, n, idx, cap); break;
        case 2: index_build_kernel<2><<<g, 256, 0, s>>>(keys, n, idx, cap); break;
        case 3: index_build_kernel<3><<<g, 256, 0, s>>>(keys, n, idx, cap); break;
        case 4: index_build_kernel<4><<<g, 256, 0, s>>>(keys, n, idx, cap); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Bytes of piece i: src[psrc[i] .. psrc[i] + (pdst[i + 1] - pdst[i])) copied
// to dst[pdst[i] ..); one CTA per piece at a time.
__global__ void __launch_bounds__(256) piece_copy_kernel(const char* __restrict__ src,
                                                         const unsigned long long* __restrict__ psrc,
                                                         const unsigned long long* __restrict__ pdst,
                                                         unsigned long long n_pieces, char* __restrict__ dst) {
    for (unsigned long long i = blockIdx.x; i < n_pieces; i += gridDim.x) {
        const unsigned long long a = psrc[i], b0 = pdst[i], len = pdst[i + 1] - b0;
        for (unsigned long long j = threadIdx.x; j < len; j += 256) dst[b0 + j] = src[a + j];
    }
}

cudaError_t launch_piece_copy(const char* src, const unsigned long long* psrc, const unsigned long long* pdst,
                              unsigned long long n_pieces, char* dst, int num_sms, cudaStream_t s) {
    if (n_pieces == 0) return cudaSuccess;
    const unsigned long long g = n_pieces < (unsigned long long)num_sms * 16 ? n_pieces : (unsigned long long)num_sms * 16;
    piece_copy_kernel<<<(unsigned)g, 256, 0, s>>>(src, psrc, pdst, n_pieces, dst);
    return cudaGetLastError();
}

cudaError_t launch_merge_append(unsigned W, const unsigned long long* bkeys, const unsigned char* bcls,
                                unsigned long long bn, const unsigned* idx, unsigned long long cap,
                                unsigned long long* keys, unsigned* count, unsigned* ext, unsigned char* cls,
                                unsigned long long out_cap, unsigned long long* n_out, unsigned* status, int num_sms,
                                cudaStream_t s) {
    if (bn == 0) return cudaSuccess;
    const unsigned g = grid_of(bn, num_sms);
    switch (W) {
        case 1: merge_append_kernel<1><<<g, 256, 0, s>>>(bkeys, bcls, bn, idx, cap, keys, count, ext, cls, out_cap, n_out, status); break;
        case 2: merge_append_kernel<2><<<g, 256, 0, s>>>(bkeys, bcls, bn, idx, cap, keys, count, ext, cls, out_cap, n_out, status); break;
        case 3: merge_append_kernel<3><<<g, 256, 0, s>>>(bkeys, bcls, bn, idx, cap, keys, count, ext, cls, out_cap, n_out, status); break;
        case 4: merge_append_kernel<4><<<g, 256, 0, s>>>(bkeys, bcls, bn, idx, cap, keys, count, ext, cls, out_cap, n_out, status); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_lookup(unsigned W, const unsigned long long* q, unsigned long long n, unsigned k,
                          const unsigned* idx, unsigned long long cap, const unsigned long long* keys,
                          const unsigned* count, const unsigned* ext, const unsigned char* cls, kmer_record* out,
                          int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned g = grid_of(n, num_sms);
    switch (W) {
        case 1: lookup_kernel<1><<<g, 256, 0, s>>>(q, n, k, idx, cap, keys, count, ext, cls, out); break;
        case 2: lookup_kernel<2><<<g, 256, 0, s>>>(q, n, k, idx, cap, keys, count, ext, cls, out); break;
        case 3: lookup_kernel<3><<<g, 256, 0, s>>>(q, n, k, idx, cap, keys, count, ext, cls, out); break;
        case 4: lookup_kernel<4><<<g, 256, 0, s>>>(q, n, k, idx, cap, keys, count, ext, cls, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace kmer
