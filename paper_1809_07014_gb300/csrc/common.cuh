// Shared device definitions of the k-mer analysis library (sm_103a).
//
// Data layout in HBM
//   PackedBlock  : 32 bases of one read, 2 bits per base MSB-first
//                  (A=0, C=1, G=2, T=3, so numeric order = lexicographic
//                  order), plus an N bit and a high-quality bit per base.
//                  Every read starts on a block boundary.
//   key          : a canonical k-mer as W = ceil(2k/64) 64-bit words, word 0
//                  most significant (it holds the first 2k - 64(W-1) bits).
//   record       : one k-mer window after partitioning: W words.  Words
//                  0..W-2 are the key's head words verbatim; word W-1 (the
//                  "tail") holds the low bits of z, a bijective mix of the
//                  key's last word, with the partition bits of z removed
//                  (they are implied by the partition the record sits in),
//                  shifted left by 6, and the window's extension code in
//                  the low 6 bits (left code << 3 | right code).
//
// The partitioning is the device-wide form of the paper's owner-computes
// k-mer histogram (Sec. II-A, use case 4; Sec. II-B): a hash of the k-mer
// picks its owner (a pass, a level-1 bucket, a leaf), and each leaf is then
// counted alone in an on-chip table.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kmer {

constexpr int kMaxW = 4;
constexpr int kMaxK = 127;

struct __align__(16) PackedBlock {
    unsigned long long bases;  // base j at bits [63-2j-1, 63-2j] (MSB first)
    unsigned int nmask;        // bit j = base j is not A/C/G/T
    unsigned int hqmask;       // bit j = Phred(base j) >= quality threshold
};

// Device status word bits (latched; the host reads them after a query).
enum StatusBits : unsigned int {
    ST_L1_OVERFLOW = 1u << 0,    // a level-1 bucket got more records than its capacity
    ST_L2_OVERFLOW = 1u << 1,    // a leaf got more records than its capacity
    ST_OUT_OVERFLOW = 1u << 2,   // more survivors than the output capacity
    ST_FALLBACK_FULL = 1u << 3,  // more overflowing leaves than the fallback list holds
    ST_TABLE_FULL = 1u << 4,     // an HBM table ran out of slots
    ST_TIMEOUT = 1u << 5,        // a bounded spin gave up
    ST_COUNTER_OVERFLOW = 1u << 6,
    ST_L2_PLAN = 1u << 7,        // the level-2 planner found the leaf layout larger than the buffer
    ST_SORT_RANGE = 1u << 8,     // a radix-sort position fell outside the survivors (write skipped)
};

// Extension code of one window: left and right in {0 = none, 1..4 = A,C,G,T + 1},
// three bits each.
__host__ __device__ inline unsigned ext_code(unsigned left, unsigned right) { return (left << 3) | right; }
__host__ __device__ inline unsigned ext_left(unsigned long long tail) { return (unsigned)(tail >> 3) & 7u; }
__host__ __device__ inline unsigned ext_right(unsigned long long tail) { return (unsigned)tail & 7u; }

// ---------------------------------------------------------------- mixing
__host__ __device__ constexpr unsigned long long inv_odd(unsigned long long c) {
    unsigned long long x = c;  // Newton iteration for the inverse mod 2^64
    for (int i = 0; i < 6; ++i) x *= 2ull - c * x;
    return x;
}
constexpr unsigned long long kM1 = 0xBF58476D1CE4E5B9ull;
constexpr unsigned long long kM1i = inv_odd(kM1);
static_assert(kM1 * kM1i == 1ull, "odd inverse");

__host__ __device__ inline unsigned long long low_mask(unsigned b) {
    return b >= 64 ? ~0ull : ((1ull << b) - 1ull);
}

// Hash of the head words (words 0..W-2) that is xored into the last word
// before the multiply, so that z depends on the whole key.
template <int W>
__host__ __device__ inline unsigned long long head_hash(const unsigned long long (&w)[W]) {
    unsigned long long h = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int i = 0; i < W - 1; ++i) {
        h ^= w[i];
        h ^= h >> 31;
        h *= 0x94D049BB133111EBull;
        h ^= h >> 29;
    }
    return W > 1 ? h : 0ull;
}

// Geometry of one analysis: k-mer words, mixing width and partition bits.
struct Geometry {
    unsigned k, W;
    unsigned hb;   // bits in key word 0
    unsigned bt;   // bits of z (2k for W == 1, else 64)
    unsigned ps;   // pass bits (top of z)
    unsigned p1;   // level-1 bucket bits
    unsigned p2;   // level-2 (leaf within bucket) bits
    __host__ __device__ unsigned zl_bits() const { return bt - ps - p1; }  // bits of z kept in the record
};

// z of a key: a bijection of its last word times an odd constant modulo 2^bt,
// whose top bits (the partition) depend on every bit through the carries.
// One word (k <= 31, bt = 2k): the key itself.  Several words (bt = 64): the
// last word xored with a hash of the head words, so that z depends on the
// whole key.
template <int W>
__host__ __device__ inline unsigned long long key_to_z(const unsigned long long (&key)[W], unsigned bt) {
    return W == 1 ? (key[0] * kM1) & low_mask(bt) : (key[W - 1] ^ head_hash<W>(key)) * kM1;
}
// Recover the key's last word from z and the head words.
template <int W>
__host__ __device__ inline unsigned long long z_to_tail(unsigned long long z, const unsigned long long (&key)[W],
                                                     unsigned bt) {
    return W == 1 ? (z * kM1i) & low_mask(bt) : ((z * kM1i) ^ head_hash<W>(key));
}

// ------------------------------------------------------- job description
// Everything one k-mer analysis needs on the device, for one pass.
struct Job {
    // packed reads
    const PackedBlock* blocks;
    const unsigned long long* blk_off;  // n_reads + 1 block offsets
    const unsigned long long* offsets;  // n_reads + 1 base offsets
    unsigned long long n_reads;
    Geometry g;
    unsigned pass;
    // level-1 buckets (P1 = 1 << g.p1).  The level-2 stages may take a window
    // of them (a wave): buckets bucket0 .. bucket0 + n_buckets - 1, with the
    // per-bucket arrays below starting at bucket0 and the level-2 arrays
    // holding that window only; n_buckets = 0 means all P1 buckets.
    unsigned bucket0, n_buckets;
    unsigned long long* l1_rec;            // records, W words each
    const unsigned long long* l1_start;    // record index of each bucket
    const unsigned long long* l1_cap;      // capacity (records) of each bucket
    unsigned long long* l1_fill;           // records offered to each bucket
    // level-2 leaves (P = 1 << (p1 + p2)); unused when p2 == 0
    unsigned long long* l2_rec;
    unsigned long long* l2_base;           // per bucket: record index of its first leaf
    unsigned int* l2_leafcap;              // per bucket: capacity of each of its leaves
    unsigned long long* l2_fill;           // per leaf: records offered
    const unsigned long long* l2_leaf_start;  // per leaf + 1: exact layout (after an overflow) or null
    unsigned long long* tile_prefix;       // per bucket + 1: level-2 tiles before it
    unsigned long long l2_capacity;        // records the level-2 buffer holds (uniform layout check)
    // outputs (survivors)
    unsigned long long* out_keys;  // n * W
    unsigned int* out_count;
    unsigned int* out_ext;         // n * 8
    unsigned char* out_cls;        // n * 2
    unsigned long long out_cap;
    unsigned long long* out_n;     // survivors written (atomic)
    // leaves whose keys did not fit their table, counted again in key ranges
    unsigned int* split_list;
    unsigned int* split_n;
    unsigned int split_cap;
    // key ranges (fallback_entry) handed to the HBM-table fallback
    unsigned int* fb_list;
    unsigned int* fb_n;
    unsigned int fb_cap;
    // Bloom gate (gate.cu): F2, 2^gate_bits words; null = every window is emitted
    const unsigned long long* gate;
    unsigned gate_bits;
    // classification
    unsigned min_count, ext_mode, t_base, err_num, err_den, t_ext;
    // sizing: level-2 leaf capacity = mean * l2_slack_num / 256 + 256 records;
    // leaf table slots = records * table_ratio_num / 65536 + 512 (capped)
    unsigned l2_slack_num;
    unsigned table_ratio_num;
    // status and statistics
    unsigned int* status;
    unsigned long long* stats;  // [0] windows counted, [1] distinct keys, [2] records emitted,
                                // [3] leaves counted in rounds, [4] heavy sub-bins walked in key ranges
};

// ------------------------------------------------------------ classify
// One side of a k-mer: tallies n[4], count d.  Codes 0..3 = unique base,
// 4 = fork, 5 = dead end.  Mode 0 is the depth-adaptive rule of Sec. II-C
// (extend iff at most t_hq = max(t_base, e*d) extensions contradict the most
// common one, e = err_num/err_den, compared exactly); mode 1 the static
// high-quality-extension count t_ext of Sec. II-B.
__device__ inline unsigned char classify_side(const unsigned (&n)[4], unsigned d, const Job& j) {
    if (j.ext_mode == 1) {
        int hq = 0, which = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (n[b] >= j.t_ext) { ++hq; which = b; }
        return hq == 0 ? 5 : (hq == 1 ? (unsigned char)which : 4);
    }
    unsigned best = 0, total = 0;
    int m = 0, ties = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        total += n[b];
        if (n[b] > best) { best = n[b]; m = b; ties = 1; }
        else if (n[b] == best) ++ties;
    }
    if (best == 0) return 5;
    if (ties > 1) return 4;
    unsigned long long alt = (unsigned long long)(total - best) * j.err_den;
    unsigned long long a = (unsigned long long)j.t_base * j.err_den;
    unsigned long long e = (unsigned long long)j.err_num * d;
    return alt <= (a > e ? a : e) ? (unsigned char)m : 4;
}

__device__ inline void set_status(const Job& j, unsigned bits) { atomicOr(j.status, bits); }

// Level-1 buckets the level-2 stages of a job take (a wave, or all of them).
__host__ __device__ inline unsigned job_buckets(const Job& j) { return j.n_buckets ? j.n_buckets : 1u << j.g.p1; }

// Index of the job that owns work unit `u`, given the exclusive prefix `off`
// (n + 1 entries) of the jobs' unit counts (jobs with no units are skipped).
__device__ __forceinline__ unsigned job_of(const unsigned long long* off, unsigned n, unsigned long long u) {
    unsigned lo = 0, hi = n - 1;
    while (lo < hi) {
        const unsigned mid = (lo + hi + 1) >> 1;
        if (off[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace kmer
