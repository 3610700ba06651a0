// Operations on canonical k-mer keys held as W 64-bit words (word 0 most
// significant, holding the first 2k - 64(W-1) bits): base access, the
// survivors' index (an open-addressing table of survivor positions), and the
// shifts that step from a k-mer to its neighbours in the de Bruijn graph.
#pragma once
#include "common.cuh"

namespace kmer {

constexpr unsigned kIdxEmpty = 0xFFFFFFFFu;

template <int W>
__device__ __forceinline__ unsigned long long key_hash(const unsigned long long (&key)[W]) {
    unsigned long long x = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        x ^= key[w];
        x *= 0xFF51AFD7ED558CCDull;
        x ^= x >> 33;
    }
    return x;
}

// Base i (0 = first, most significant) of a k-mer held as W words, word 0
// most significant.
template <int W>
__device__ __forceinline__ unsigned get_base(const unsigned long long (&key)[W], unsigned k, unsigned i) {
    const unsigned pos = 2 * (k - 1 - i);  // bit position from the least significant end
    return (unsigned)(key[W - 1 - pos / 64] >> (pos % 64)) & 3u;
}

template <int W>
__device__ __forceinline__ void set_base(unsigned long long (&key)[W], unsigned k, unsigned i, unsigned b) {
    const unsigned pos = 2 * (k - 1 - i);
    key[W - 1 - pos / 64] |= (unsigned long long)b << (pos % 64);
}

// Position of `key` among the survivors through the index, or kIdxEmpty.
template <int W>
__device__ __forceinline__ unsigned index_find(const unsigned long long (&key)[W], const unsigned* __restrict__ idx,
                                               unsigned long long cap, const unsigned long long* __restrict__ keys) {
    unsigned long long s = key_hash<W>(key) & (cap - 1);
    for (unsigned long long probe = 0; probe < cap; ++probe) {
        const unsigned p = idx[s];
        if (p == kIdxEmpty) return kIdxEmpty;
        bool same = true;
#pragma unroll
        for (int w = 0; w < W; ++w) same = same && keys[(unsigned long long)p * W + w] == key[w];
        if (same) return p;
        s = (s + 1) & (cap - 1);
    }
    return kIdxEmpty;
}

// The k-mer shifted one base to the left with base b appended (the right
// neighbour's string); hb = bits of word 0.
template <int W>
__device__ __forceinline__ void shift_in_right(unsigned long long (&x)[W], unsigned b, unsigned hb) {
#pragma unroll
    for (int w = 0; w < W - 1; ++w) x[w] = (x[w] << 2) | (x[w + 1] >> 62);
    x[W - 1] = (x[W - 1] << 2) | b;
    x[0] &= low_mask(hb);
}

// The k-mer shifted one base to the right with base b put first (the left
// neighbour's string).
template <int W>
__device__ __forceinline__ void shift_in_left(unsigned long long (&x)[W], unsigned b, unsigned hb) {
#pragma unroll
    for (int w = W - 1; w > 0; --w) x[w] = (x[w] >> 2) | (x[w - 1] << 62);
    x[0] = (x[0] >> 2) | ((unsigned long long)b << (hb - 2));
}

template <int W>
__device__ __forceinline__ void reverse_complement(const unsigned long long (&x)[W], unsigned k,
                                                   unsigned long long (&rc)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) rc[w] = 0;
    for (unsigned b = 0; b < k; ++b) set_base<W>(rc, k, k - 1 - b, 3u - get_base<W>(x, k, b));
}

// a < b, word 0 first (lexicographic order of the k-mers).
template <int W>
__device__ __forceinline__ bool key_less(const unsigned long long (&a)[W], const unsigned long long (&b)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w)
        if (a[w] != b[w]) return a[w] < b[w];
    return false;
}

}  // namespace kmer
