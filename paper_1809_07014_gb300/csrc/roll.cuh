// Steps a2 + a3: slide a k-window over one packed read, keep the forward
// k-mer and its reverse complement as W-word shift registers, and produce for
// every window without N its canonical key (the smaller of the two) and its
// extension code.  Sec. II-B: k-mers overlap by k-1 bases; the extensions are
// the bases just before and after the window in the read, kept only if they
// are A/C/G/T with Phred >= threshold (the pack step folded both tests into
// one "good" bit per base).
#pragma once
#include "common.cuh"

namespace kmer {

// HI (one word, k >= 17): the window's first base sits in the high 32 bits
// of the word, so the base leaving the window and the complement entering the
// reverse strand touch that half only.
template <int W, bool HI = false>
struct Roll {
    unsigned long long fwd[W], rc[W];
    unsigned long long gh0, gh1;  // good bits of the last 128 bases, bit m = base t-1-m
    long long last_n;             // last position holding an N (or -1)
    unsigned long long cur;       // bases of the current block, next base in the top 2 bits
    unsigned curn, curg;          // N / good bits of the current block, next base in bit 0
    uint4 nxt;                    // the block after the current one, loaded one block ahead
    unsigned out;                 // base that left the window at the last step
    const PackedBlock* blk;
    unsigned long long L;
    unsigned k, hb;
    unsigned long long topmask;

    __device__ void init(const Job& j, unsigned long long r) {
        const unsigned long long a = j.offsets[r];
        L = j.offsets[r + 1] - a;
        blk = j.blocks + j.blk_off[r];
        k = j.g.k;
        hb = j.g.hb;
        topmask = low_mask(hb);
#pragma unroll
        for (int i = 0; i < W; ++i) { fwd[i] = 0; rc[i] = 0; }
        gh0 = gh1 = 0;
        last_n = -1;
        out = 0;
        cur = 0;
        curn = curg = 0;
        nxt = L ? __ldg(reinterpret_cast<const uint4*>(blk)) : make_uint4(0, 0, 0, 0);
    }

    // Step t (0 <= t <= L).  First the window [t-k, t) is reported if t >= k
    // and it holds no N; then base t (if t < L) is shifted in.  Returns true
    // and fills key / lcode / rcode (0 = none, 1..4 = A..T) for a window.
    __device__ __forceinline__ bool step(unsigned long long t, unsigned long long (&key)[W], unsigned& lcode,
                                         unsigned& rcode) {
        unsigned b = 0, good = 0, isn = 0;
        if (t < L) {
            if ((t & 31) == 0) {
                cur = ((unsigned long long)nxt.y << 32) | nxt.x;
                curn = nxt.z;
                curg = nxt.w;
                if (t + 32 < L) nxt = __ldg(reinterpret_cast<const uint4*>(blk + (t >> 5) + 1));
            }
            b = (unsigned)(cur >> 62);
            cur <<= 2;
            isn = curn & 1u;
            curn >>= 1;
            good = curg & 1u;
            curg >>= 1;
        }
        bool emit = false;
        if (t >= k && last_n < (long long)(t - k)) {
            emit = true;
            // the history holds zeros before the read's first base, so the
            // first window finds no left extension, and `good` is 0 past the end
            const unsigned lgood = k < 64 ? (unsigned)(gh0 >> k) & 1u : (unsigned)(gh1 >> (k - 64)) & 1u;
            unsigned lc = lgood ? out + 1 : 0;
            unsigned rcd = good ? b + 1 : 0;
            // canonical: the lexicographically smaller of forward and reverse complement
            bool flip = false;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (fwd[w] != rc[w]) { flip = rc[w] < fwd[w]; break; }
            }
#pragma unroll
            for (int w = 0; w < W; ++w) key[w] = flip ? rc[w] : fwd[w];
            if (flip) {  // the key reads the other strand: swap sides, complement bases
                const unsigned nl = rcd ? 5 - rcd : 0, nr = lc ? 5 - lc : 0;
                lc = nl;
                rcd = nr;
            }
            lcode = lc;
            rcode = rcd;
        }
        if (t < L) {
            out = (unsigned)(fwd[0] >> (hb - 2)) & 3u;
#pragma unroll
            for (int w = 0; w < W - 1; ++w) fwd[w] = (fwd[w] << 2) | (fwd[w + 1] >> 62);
            fwd[W - 1] = (fwd[W - 1] << 2) | b;
            fwd[0] &= topmask;
#pragma unroll
            for (int w = W - 1; w > 0; --w) rc[w] = (rc[w] >> 2) | (rc[w - 1] << 62);
            rc[0] = (rc[0] >> 2) | ((unsigned long long)(3u - b) << (hb - 2));
            gh1 = (gh1 << 1) | (gh0 >> 63);
            gh0 = (gh0 << 1) | good;
            if (isn) last_n = (long long)t;
        }
        return emit;
    }
};

// k <= 31: the whole k-mer fits one word; positions and the quality history
// fit 32 bits (reads are shorter than 2^31 bases).
template <bool HI>
struct Roll<1, HI> {
    unsigned long long fwd, rc, mask, cur;
    unsigned curn, curg, gh, out, L, k, sh;
    int first_ok;  // first step whose window holds no N: last N position + k + 1
    uint4 nxt;
    const PackedBlock* blk;

    __device__ void init(const Job& j, unsigned long long r) {
        const unsigned long long a = j.offsets[r];
        L = (unsigned)(j.offsets[r + 1] - a);
        blk = j.blocks + j.blk_off[r];
        k = j.g.k;
        sh = 2 * k - 2;
        mask = low_mask(2 * k);
        fwd = rc = cur = 0;
        curn = curg = gh = out = 0;
        first_ok = (int)k;
        nxt = L ? __ldg(reinterpret_cast<const uint4*>(blk)) : make_uint4(0, 0, 0, 0);
    }

    __device__ __forceinline__ bool step(unsigned long long t64, unsigned long long (&key)[1], unsigned& lcode,
                                         unsigned& rcode) {
        const unsigned t = (unsigned)t64;
        const bool in = t < L;
        unsigned b = 0, good = 0, isn = 0;
        if (in) {
            if ((t & 31) == 0) {
                cur = ((unsigned long long)nxt.y << 32) | nxt.x;
                curn = nxt.z;
                curg = nxt.w;
                if (t + 32 < L) nxt = __ldg(reinterpret_cast<const uint4*>(blk + (t >> 5) + 1));
            }
            b = (unsigned)(cur >> 62);
            cur <<= 2;
            isn = curn & 1u;
            curn >>= 1;
            good = curg & 1u;
            curg >>= 1;
        }
        bool emit = false;
        if ((int)t >= first_ok) {
            emit = true;
            // gh is zero before the first base and `good` is 0 past the end
            unsigned lc = ((gh >> k) & 1u) ? out + 1 : 0;
            unsigned rcd = good ? b + 1 : 0;
            const bool flip = rc < fwd;
            key[0] = flip ? rc : fwd;
            if (flip) {  // the key reads the other strand: swap sides, complement bases
                const unsigned nl = rcd ? 5 - rcd : 0, nr = lc ? 5 - lc : 0;
                lc = nl;
                rcd = nr;
            }
            lcode = lc;
            rcode = rcd;
        }
        if (in) {
            if (HI) {
                out = ((unsigned)(fwd >> 32) >> (sh - 32)) & 3u;
                rc = (rc >> 2) | ((unsigned long long)((3u - b) << (sh - 32)) << 32);
            } else {
                out = (unsigned)(fwd >> sh) & 3u;
                rc = (rc >> 2) | ((unsigned long long)(3u - b) << sh);
            }
            fwd = ((fwd << 2) | b) & mask;
            gh = (gh << 1) | good;
            if (isn) first_ok = (int)(t + k + 1);
        }
        return emit;
    }
};

// Record of one window (words 0..W-2 = head words, word W-1 = tail) and its
// level-1 bucket; returns false when the window belongs to another pass.
template <int W>
__device__ __forceinline__ bool make_record(const Geometry& g, unsigned pass, const unsigned long long (&key)[W],
                                            unsigned lcode, unsigned rcode, unsigned long long (&rec)[W],
                                            unsigned& bucket) {
    const unsigned long long z = key_to_z<W>(key, g.bt);
    if (g.ps && (unsigned)(z >> (g.bt - g.ps)) != pass) return false;
    const unsigned zb = g.zl_bits();
    bucket = g.p1 ? (unsigned)(z >> zb) & ((1u << g.p1) - 1u) : 0u;
#pragma unroll
    for (int w = 0; w < W - 1; ++w) rec[w] = key[w];
    rec[W - 1] = ((z & low_mask(zb)) << 6) | ext_code(lcode, rcode);
    return true;
}

// Bloom-gate hash of a canonical key (gate.cu): the 64-bit finaliser of
// MurmurHash3 applied to the last word xored with a hash of the head words.
template <int W>
__device__ __forceinline__ unsigned long long gate_hash(const unsigned long long (&key)[W]) {
    unsigned long long h = key[W - 1] ^ head_hash<W>(key) ^ 0x2545F4914F6CDD1Dull;
    h ^= h >> 33;
    h *= 0xFF51AFD7ED558CCDull;
    h ^= h >> 33;
    h *= 0xC4CEB9FE1A85EC53ull;
    h ^= h >> 33;
    return h;
}

// The filter word (top log2_words bits of the hash) and four bits within it
// (four 6-bit fields of the low bits).
struct GateProbe {
    unsigned long long word, mask;
};
__device__ __forceinline__ GateProbe gate_probe(unsigned long long h, unsigned log2_words) {
    GateProbe p;
    p.word = log2_words ? h >> (64 - log2_words) : 0ull;
    p.mask = (1ull << (h & 63)) | (1ull << ((h >> 6) & 63)) | (1ull << ((h >> 12) & 63)) | (1ull << ((h >> 18) & 63));
    return p;
}

// The key is in the gate's filter (every bit of its probe set).
template <int W>
__device__ __forceinline__ bool gate_has(const unsigned long long* f, unsigned log2_words,
                                         const unsigned long long (&key)[W]) {
    const GateProbe p = gate_probe(gate_hash<W>(key), log2_words);
    return (__ldg(f + p.word) & p.mask) == p.mask;
}

// z of a record held in a known pass and level-1 bucket.
__device__ __forceinline__ unsigned long long record_z(const Geometry& g, unsigned pass, unsigned bucket,
                                                       unsigned long long tail) {
    const unsigned zb = g.zl_bits();
    unsigned long long z = tail >> 6;
    if (g.p1) z |= (unsigned long long)bucket << zb;
    if (g.ps) z |= (unsigned long long)pass << (g.bt - g.ps);
    return z;
}

}  // namespace kmer
