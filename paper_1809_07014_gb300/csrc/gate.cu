// Bloom-filter gate (Sec. II-B): k-mers seen only once are, at these error
// rates, mostly sequencing errors, and the paper keeps them out of the
// distributed hash tables with Bloom filters so that they do not blow up its
// memory.  Here the gate runs before the scatter: every window's canonical
// key is added to filter F1, and a key found already present in F1 (seen
// before, or a false positive) is added to filter F2.  The scatter then emits
// only windows whose key is in F2.
//
// Exact for min_count >= 2: a key seen twice or more has every bit of its
// probe set in F1 by its first sighting before any later sighting's atomicOr
// reads F1 (the atomics are linearizable), so that later sighting puts it
// into F2, and every one of its windows passes the scatter's test.  A key
// seen once passes only as a false positive, and is then counted exactly
// (count 1) and dropped by the count filter.
//
// Filters are blocked: a key touches one 64-bit word of each, setting four
// bits, with one atomicOr per filter.
#include "kernels.h"
#include "roll.cuh"

namespace kmer {

template <int W, bool HI>
__global__ void __launch_bounds__(256) gate_kernel(const Job j, unsigned long long* __restrict__ f1,
                                                   unsigned long long* __restrict__ f2, const unsigned log2_words,
                                                   unsigned long long* __restrict__ counts) {
    const unsigned long long r = blockIdx.x * 256ull + threadIdx.x;
    unsigned windows = 0, first = 0, second = 0;
    if (r < j.n_reads) {
        Roll<W, HI> roll;
        roll.init(j, r);
        for (unsigned long long t = 0; t <= roll.L; ++t) {
            unsigned long long key[W];
            unsigned lc, rc;
            if (!roll.step(t, key, lc, rc)) continue;
            ++windows;
            const GateProbe p = gate_probe(gate_hash<W>(key), log2_words);
            const unsigned long long o1 = atomicOr(f1 + p.word, p.mask);
            if ((o1 & p.mask) != p.mask) {
                ++first;  // first sighting (or a false positive of F1)
            } else if ((__ldcg(f2 + p.word) & p.mask) != p.mask) {
                const unsigned long long o2 = atomicOr(f2 + p.word, p.mask);
                if ((o2 & p.mask) != p.mask) ++second;  // a key entering F2
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        windows += __shfl_xor_sync(0xffffffffu, windows, o);
        first += __shfl_xor_sync(0xffffffffu, first, o);
        second += __shfl_xor_sync(0xffffffffu, second, o);
    }
    if ((threadIdx.x & 31) == 0 && windows) {
        atomicAdd(counts + 0, (unsigned long long)windows);
        atomicAdd(counts + 1, (unsigned long long)first);
        atomicAdd(counts + 2, (unsigned long long)second);
    }
}

template <int W, bool HI>
static cudaError_t launch_gate_w(const Job& j, unsigned long long* f1, unsigned long long* f2, unsigned log2_words,
                                 unsigned long long* counts, cudaStream_t s) {
    if (j.n_reads == 0) return cudaSuccess;
    const unsigned long long grid = (j.n_reads + 255) / 256;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    gate_kernel<W, HI><<<(unsigned)grid, 256, 0, s>>>(j, f1, f2, log2_words, counts);
    return cudaGetLastError();
}

cudaError_t launch_gate(const Job& j, unsigned long long* f1, unsigned long long* f2, unsigned log2_words,
                        unsigned long long* counts, cudaStream_t s) {
    switch (j.g.W) {
        case 1:
            return j.g.k >= 17 ? launch_gate_w<1, true>(j, f1, f2, log2_words, counts, s)
                               : launch_gate_w<1, false>(j, f1, f2, log2_words, counts, s);
        case 2: return launch_gate_w<2, false>(j, f1, f2, log2_words, counts, s);
        case 3: return launch_gate_w<3, false>(j, f1, f2, log2_words, counts, s);
        case 4: return launch_gate_w<4, false>(j, f1, f2, log2_words, counts, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kmer
