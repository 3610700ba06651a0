// De Bruijn graph traversal (Sec. II-C): contigs are the paths formed by
// k-mers with unique high-quality extensions.  The graph is held implicitly
// by the survivors and their two-letter codes (Sec. II-C: key + code name the
// neighbours); here it is walked with list ranking instead of the paper's
// one-walker-per-seed traversal over a distributed hash table.
//
// A vertex is a survivor whose two sides are both UNIQUE.  It has two ports,
// left (0) and right (1) of its stored orientation.  Read in an orientation x,
// it names its right neighbour y = x[1..k) + r(x); the two are joined when y's
// canonical form is another vertex whose own left base, read in y's
// orientation, is x[0] (each names the other).  A k-mer followed by its own
// reverse complement (a hairpin) is joined to nothing there.  Each port has at
// most one partner, so the vertices form chains and rings:
//
//  1. links: one kernel looks up both neighbours of every vertex in the
//     survivors' index and keeps mutual ones (port -> partner port);
//  2. list ranking, for every port the end reached by walking out of it and
//     the number of steps, by a ruling set: about one port in 16 (by a hash)
//     and every path start is a ruler; each ruler walks to the next ruler or
//     the path's end, marking the ports it passes with itself and their
//     distance from it; the rulers are then ranked by pointer jumping (in
//     place, over the rulers not yet at an end: a port may read a partner's
//     walk from this round or the last, both true statements about the path),
//     and every port takes its ruler's result less its distance.  The work is
//     about one random access per port instead of one per port and round;
//  3. rings (ports whose walk never ends) are cut before their smallest
//     canonical k-mer (found by doubling a running minimum around the ring),
//     and only their ports are ranked again;
//  4. every chain is written from its end with the smaller index: the end's
//     k-mer, then one base per later vertex at its distance from the end; the
//     chains' lengths are scanned into offsets;
//  5. every contig is turned into the smaller of itself and its reverse
//     complement, in chunks of 256 positions spread over the whole grid (a
//     contig can be millions of bases long).
#include "kernels.h"
#include "keyops.cuh"

namespace kmer {

constexpr unsigned kNoPort = 0xFFFFFFFFu;

__device__ __forceinline__ bool is_vertex(const unsigned char* cls, unsigned long long i) {
    return cls[2 * i] < 4 && cls[2 * i + 1] < 4;
}

// link[2i + p]: partner port (2j + q) of vertex i's port p, or kNoPort.
template <int W>
__global__ void __launch_bounds__(256) links_kernel(const unsigned long long* __restrict__ keys,
                                                    const unsigned char* __restrict__ cls, unsigned long long n,
                                                    unsigned k, const unsigned* __restrict__ idx,
                                                    unsigned long long cap, unsigned* __restrict__ link) {
    const unsigned hb = 2 * k - 64 * (W - 1);
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * 256) {
        unsigned l0 = kNoPort, l1 = kNoPort;
        if (is_vertex(cls, i)) {
            unsigned long long x[W], rc[W];
#pragma unroll
            for (int w = 0; w < W; ++w) x[w] = keys[i * W + w];
            reverse_complement<W>(x, k, rc);
            const unsigned first = get_base<W>(x, k, 0), last = get_base<W>(x, k, k - 1);
            for (unsigned p = 0; p < 2; ++p) {
                // the neighbour's string y and its reverse complement
                unsigned long long y[W], yr[W];
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    y[w] = x[w];
                    yr[w] = rc[w];
                }
                const unsigned b = cls[2 * i + p];
                if (p == 1) {
                    shift_in_right<W>(y, b, hb);
                    shift_in_left<W>(yr, 3u - b, hb);
                } else {
                    shift_in_left<W>(y, b, hb);
                    shift_in_right<W>(yr, 3u - b, hb);
                }
                const bool flip = key_less<W>(yr, y);
                const unsigned j = index_find<W>(flip ? yr : y, idx, cap, keys);
                if (j == kIdxEmpty || j == i || !is_vertex(cls, j)) continue;
                // y's base on the side facing x, read in y's orientation
                bool mutual;
                unsigned q;
                if (p == 1) {  // x -> y: y's left base must be x's first
                    const unsigned ly = flip ? 3u - cls[2ull * j + 1] : cls[2ull * j];
                    mutual = ly == first;
                    q = flip ? 1u : 0u;
                } else {  // y -> x: y's right base must be x's last
                    const unsigned ry = flip ? 3u - cls[2ull * j] : cls[2ull * j + 1];
                    mutual = ry == last;
                    q = flip ? 0u : 1u;
                }
                if (mutual) (p ? l1 : l0) = (unsigned)(2 * j + q);
            }
        }
        link[2 * i] = l0;
        link[2 * i + 1] = l1;
    }
}

// Walk state of a port P, one 64-bit word (dist << 32 | at), read and written
// whole: after dist steps out of P the walk stands at port-code `at` (a vertex
// and the port it would leave by next); dist 0 = P has no partner (the walk
// ends at once).
__device__ __forceinline__ unsigned long long walk_pack(unsigned at, unsigned dist) {
    return (unsigned long long)dist << 32 | at;
}
__device__ __forceinline__ unsigned walk_at(unsigned long long w) { return (unsigned)w; }
__device__ __forceinline__ unsigned walk_dist(unsigned long long w) { return (unsigned)(w >> 32); }

// Appends val to list when pred holds: one atomic per warp.
__device__ __forceinline__ void append_if(bool pred, unsigned val, unsigned* list, unsigned* count) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(act, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// First walks of the ports of a list (the rings, after their cut): one step to
// the partner's other port; linked ports go to the active list.
__global__ void __launch_bounds__(256) walk_reinit_kernel(const unsigned* __restrict__ link,
                                                          const unsigned* __restrict__ list,
                                                          const unsigned* __restrict__ list_n,
                                                          unsigned long long* __restrict__ wk, unsigned* act,
                                                          unsigned* cnt) {
    const unsigned n = *list_n;
    for (unsigned i = blockIdx.x * 256u + threadIdx.x; i < n; i += gridDim.x * 256u) {
        const unsigned P = list[i], L = link[P];
        wk[P] = L == kNoPort ? walk_pack(P, 0u) : walk_pack(L ^ 1u, 1u);
        append_if(L != kNoPort, P, act, cnt);
    }
}

// One round of pointer jumping over the active ports, in place.  A port
// whose walk stands at an end leaves the list; so does one whose walk reached
// cap_dist (it goes round a ring).
__global__ void __launch_bounds__(256) walk_jump_kernel(unsigned long long* wk, const unsigned* __restrict__ act_in,
                                                        const unsigned* __restrict__ cnt_in, unsigned cap_dist,
                                                        unsigned* act_out, unsigned* cnt_out) {
    const unsigned n = *cnt_in;
    for (unsigned i = blockIdx.x * 256u + threadIdx.x; i < n; i += gridDim.x * 256u) {
        const unsigned P = act_in[i];
        const unsigned long long w = __ldcg(wk + P);
        const unsigned long long f = __ldcg(wk + walk_at(w));
        bool keep = false;
        if (walk_dist(f)) {
            const unsigned long long d = (unsigned long long)walk_dist(w) + walk_dist(f);
            __stcg(wk + P, walk_pack(walk_at(f), d > cap_dist ? cap_dist : (unsigned)d));
            keep = d < cap_dist;
        }
        append_if(keep, P, act_out, cnt_out);
    }
}

// Rulers: one port in 16 by a hash of its code, and every path start.
__device__ __forceinline__ bool sampled_port(unsigned P) { return ((P * 2654435761u) >> 28) == 0u; }

// Every ruler walks to the next ruler or to its path's end: owner[V] and
// off[V] of each port V it passes (itself included) name it and V's distance
// from it; rw[R] = (next ruler or end port, steps), and rw[E] = (E, 0) for
// every end port E.  Rulers that have not reached an end go to the active
// list.  Ports on rings without a ruler keep owner kNoPort.  A walk is
// bounded by the number of ports (it cannot be longer unless the links were
// not mutual), and one that gives up is counted in *err.
__global__ void __launch_bounds__(256) ruler_walk_kernel(const unsigned* __restrict__ link, unsigned long long ports,
                                                         unsigned* __restrict__ owner, unsigned* __restrict__ off,
                                                         unsigned long long* __restrict__ rw, unsigned* act,
                                                         unsigned* cnt, unsigned* err) {
    for (unsigned long long P64 = blockIdx.x * 256ull + threadIdx.x; P64 < ports;
         P64 += (unsigned long long)gridDim.x * 256) {
        const unsigned P = (unsigned)P64;
        const unsigned L = link[P];
        if (L == kNoPort) rw[P] = walk_pack(P, 0u);
        const bool ruler = link[P ^ 1u] == kNoPort || sampled_port(P);  // a path start has no predecessor
        bool active = false;
        if (ruler) {
            owner[P] = P;
            off[P] = 0;
            if (L != kNoPort) {
                unsigned cur = L ^ 1u, steps = 1;
                for (;;) {
                    if (sampled_port(cur)) break;  // the next ruler (only path starts lack a predecessor)
                    owner[cur] = P;
                    off[cur] = steps;
                    const unsigned nl = link[cur];
                    if (nl == kNoPort) break;  // the path's end
                    if (steps >= ports) {
                        atomicAdd(err, 1u);
                        break;
                    }
                    cur = nl ^ 1u;
                    ++steps;
                }
                // either a ruler (its own walk continues from there) or an end port
                rw[P] = walk_pack(cur, steps);
                active = true;
            }
        }
        append_if(active, P, act, cnt);
    }
}

// Every port's walk from its ruler's: the same end, less the distance from
// the ruler; ports on rings get cap_dist.
__global__ void __launch_bounds__(256) ruler_final_kernel(const unsigned* __restrict__ link, unsigned long long ports,
                                                          const unsigned* __restrict__ owner,
                                                          const unsigned* __restrict__ off,
                                                          const unsigned long long* __restrict__ rw, unsigned cap_dist,
                                                          unsigned long long* __restrict__ wk) {
    for (unsigned long long P = blockIdx.x * 256ull + threadIdx.x; P < ports; P += (unsigned long long)gridDim.x * 256) {
        const unsigned R = owner[P];
        if (R == kNoPort) {  // a ring with no ruler
            wk[P] = walk_pack(link[P] ^ 1u, cap_dist);
            continue;
        }
        const unsigned long long w = rw[R];
        const unsigned d = walk_dist(w);
        wk[P] = d >= cap_dist ? walk_pack(walk_at(w), cap_dist) : walk_pack(walk_at(w), d - off[P]);
    }
}

// Rings: per port P of a ring vertex, the smallest vertex (by key) among the
// 2^r vertices met walking out of P, and where that walk stands; doubled like
// the walks.  Once 2^r passes a ring's length every port of it holds the
// ring's smallest vertex.  The ring ports go to a list; only they are read.
__global__ void __launch_bounds__(256) ring_init_kernel(const unsigned long long* __restrict__ wk,
                                                        unsigned long long ports, unsigned cap_dist,
                                                        const unsigned* __restrict__ link, unsigned* __restrict__ rmin,
                                                        unsigned long long* __restrict__ step, unsigned* ring,
                                                        unsigned* ring_n) {
    for (unsigned long long P = blockIdx.x * 256ull + threadIdx.x; P < ports; P += (unsigned long long)gridDim.x * 256) {
        const bool on_ring = walk_dist(wk[P]) >= cap_dist;
        if (on_ring) {
            rmin[P] = (unsigned)(P >> 1);
            step[P] = walk_pack(link[P] ^ 1u, 1u);
        }
        append_if(on_ring, (unsigned)P, ring, ring_n);
    }
}

template <int W>
__global__ void __launch_bounds__(256) ring_double_kernel(const unsigned* __restrict__ rmin_in,
                                                          const unsigned long long* __restrict__ step_in,
                                                          const unsigned* __restrict__ ring,
                                                          const unsigned* __restrict__ ring_n,
                                                          const unsigned long long* __restrict__ keys,
                                                          unsigned* __restrict__ rmin_out,
                                                          unsigned long long* __restrict__ step_out) {
    const unsigned n = *ring_n;
    for (unsigned i = blockIdx.x * 256u + threadIdx.x; i < n; i += gridDim.x * 256u) {
        const unsigned P = ring[i];
        unsigned m = rmin_in[P];
        const unsigned at = walk_at(step_in[P]);
        const unsigned mv = rmin_in[at];  // the next 2^r vertices, from where the walk stands
        unsigned long long a[W], b[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            a[w] = keys[(unsigned long long)m * W + w];
            b[w] = keys[(unsigned long long)mv * W + w];
        }
        if (key_less<W>(b, a)) m = mv;
        rmin_out[P] = m;
        step_out[P] = walk_pack(walk_at(step_in[at]), 0u);
    }
}

// Cut every ring before its smallest vertex i: drop the link of i's port 0
// and its partner's (i's port 1 is on the list and names i as the minimum).
__global__ void __launch_bounds__(256) ring_cut_kernel(const unsigned* __restrict__ rmin,
                                                       const unsigned* __restrict__ ring,
                                                       const unsigned* __restrict__ ring_n, unsigned* __restrict__ link) {
    const unsigned n = *ring_n;
    for (unsigned j = blockIdx.x * 256u + threadIdx.x; j < n; j += gridDim.x * 256u) {
        const unsigned P = ring[j], i = P >> 1;
        if (!(P & 1u) || rmin[P] != i) continue;
        const unsigned L = link[2 * i];
        if (L != kNoPort) link[L] = kNoPort;
        link[2 * i] = kNoPort;
    }
}

// Chain of vertex i: its two ends, distances, head (the end with the smaller
// index) and i's place.
__device__ __forceinline__ void chain_of(const unsigned long long* wk, unsigned i, unsigned& head, unsigned& pos,
                                         bool& fwd, unsigned& m) {
    const unsigned long long a = wk[2 * (unsigned long long)i], b = wk[2 * (unsigned long long)i + 1];
    const unsigned h0 = walk_dist(a) ? walk_at(a) >> 1 : i, h1 = walk_dist(b) ? walk_at(b) >> 1 : i;
    m = walk_dist(a) + walk_dist(b) + 1;
    if (h0 <= h1) {  // walking from the head reaches i through its port 0: i read as stored
        head = h0;
        pos = walk_dist(a);
        fwd = true;
    } else {
        head = h1;
        pos = walk_dist(b);
        fwd = false;
    }
}

// len[i] = bases of i's contig if i is a head, else 0.
__global__ void __launch_bounds__(256) chain_len_kernel(const unsigned long long* __restrict__ wk,
                                                        const unsigned char* __restrict__ cls, unsigned long long n,
                                                        unsigned k, unsigned long long* __restrict__ len) {
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * 256) {
        unsigned long long L = 0;
        if (is_vertex(cls, i)) {
            unsigned head, pos, m;
            bool fwd;
            chain_of(wk, (unsigned)i, head, pos, fwd, m);
            if (head == i) L = (unsigned long long)m + k - 1;
        }
        len[i] = L;
    }
}

// Bases of every contig: the head's k-mer (in the orientation that leaves
// by its linked port), then each later vertex's last base at its distance.
template <int W>
__global__ void __launch_bounds__(256) chain_write_kernel(const unsigned long long* __restrict__ wk,
                                                          const unsigned char* __restrict__ cls,
                                                          const unsigned long long* __restrict__ keys,
                                                          unsigned long long n, unsigned k,
                                                          const unsigned long long* __restrict__ off,
                                                          char* __restrict__ out) {
    const char kBase[4] = {'A', 'C', 'G', 'T'};
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * 256) {
        if (!is_vertex(cls, i)) continue;
        unsigned head, pos, m;
        bool fwd;
        chain_of(wk, (unsigned)i, head, pos, fwd, m);
        unsigned long long x[W];
#pragma unroll
        for (int w = 0; w < W; ++w) x[w] = keys[i * W + w];
        char* c = out + off[head];
        if (head == i) {
            // the head leaves by port 1 (read as stored) unless only its port 0 is linked
            const bool stored = m == 1 || walk_dist(wk[2 * i + 1]) > 0;
            for (unsigned b = 0; b < k; ++b)
                c[b] = stored ? kBase[get_base<W>(x, k, b)] : kBase[3u - get_base<W>(x, k, k - 1 - b)];
        } else {
            c[pos + k - 1] = fwd ? kBase[get_base<W>(x, k, k - 1)] : kBase[3u - get_base<W>(x, k, 0)];
        }
    }
}

__device__ __forceinline__ char comp_base(char b) {
    return b == 'A' ? 'T' : (b == 'C' ? 'G' : (b == 'G' ? 'C' : 'A'));
}

constexpr unsigned kCanonChunk = 256;  // positions of a contig's first half per work item

// chunks[c] = work items of contig c: its first ceil(L / 2) positions in
// chunks of kCanonChunk; first[c] = no difference found yet.
__global__ void __launch_bounds__(256) canon_chunks_kernel(const unsigned long long* __restrict__ coff,
                                                           unsigned long long nc,
                                                           unsigned long long* __restrict__ chunks,
                                                           unsigned long long* __restrict__ first) {
    for (unsigned long long c = blockIdx.x * 256ull + threadIdx.x; c < nc; c += (unsigned long long)gridDim.x * 256) {
        const unsigned long long half = (coff[c + 1] - coff[c] + 1) / 2;
        chunks[c] = (half + kCanonChunk - 1) / kCanonChunk;
        first[c] = ~0ull;
    }
}

// Work item t: its contig (the last c with cstart[c] <= t) and chunk.
__device__ __forceinline__ unsigned long long item_contig(const unsigned long long* cstart, unsigned long long nc,
                                                          unsigned long long t) {
    unsigned long long lo = 0, hi = nc;  // cstart[lo] <= t < cstart[hi]
    while (hi - lo > 1) {
        const unsigned long long mid = (lo + hi) / 2;
        if (cstart[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// first[c] = the first position a of contig c where c[a] differs from its
// reverse complement's a-th base, complement(c[L - 1 - a]).
__global__ void __launch_bounds__(256) canon_diff_kernel(const unsigned long long* __restrict__ coff,
                                                         const unsigned long long* __restrict__ cstart,
                                                         unsigned long long nc, unsigned long long items,
                                                         const char* __restrict__ out,
                                                         unsigned long long* __restrict__ first) {
    for (unsigned long long t = blockIdx.x * 256ull + threadIdx.x; t < items; t += (unsigned long long)gridDim.x * 256) {
        const unsigned long long c = item_contig(cstart, nc, t);
        const unsigned long long b0 = coff[c], L = coff[c + 1] - b0, half = (L + 1) / 2;
        const unsigned long long a0 = (t - cstart[c]) * kCanonChunk;
        const unsigned long long a1 = a0 + kCanonChunk < half ? a0 + kCanonChunk : half;
        for (unsigned long long a = a0; a < a1; ++a)
            if (comp_base(out[b0 + L - 1 - a]) != out[b0 + a]) {
                atomicMin(first + c, a);
                break;
            }
    }
}

// Whether each contig is replaced by its reverse complement: smaller at the
// first difference (decided before any base moves).
__global__ void __launch_bounds__(256) canon_decide_kernel(const unsigned long long* __restrict__ coff,
                                                           unsigned long long nc, const char* __restrict__ out,
                                                           unsigned long long* __restrict__ first) {
    for (unsigned long long c = blockIdx.x * 256ull + threadIdx.x; c < nc; c += (unsigned long long)gridDim.x * 256) {
        const unsigned long long f = first[c];
        if (f == ~0ull) continue;  // the contig is its own reverse complement
        const unsigned long long b0 = coff[c], L = coff[c + 1] - b0;
        if (!(comp_base(out[b0 + L - 1 - f]) < out[b0 + f])) first[c] = ~0ull;
    }
}

// Contigs to replace: the pair of positions (a, L - 1 - a) swap, complemented.
__global__ void __launch_bounds__(256) canon_flip_kernel(const unsigned long long* __restrict__ coff,
                                                         const unsigned long long* __restrict__ cstart,
                                                         unsigned long long nc, unsigned long long items,
                                                         const unsigned long long* __restrict__ first,
                                                         char* __restrict__ out) {
    for (unsigned long long t = blockIdx.x * 256ull + threadIdx.x; t < items; t += (unsigned long long)gridDim.x * 256) {
        const unsigned long long c = item_contig(cstart, nc, t);
        if (first[c] == ~0ull) continue;  // kept as it is
        const unsigned long long b0 = coff[c], L = coff[c + 1] - b0, half = (L + 1) / 2;
        const unsigned long long a0 = (t - cstart[c]) * kCanonChunk;
        const unsigned long long a1 = a0 + kCanonChunk < half ? a0 + kCanonChunk : half;
        for (unsigned long long a = a0; a < a1; ++a) {
            const char x = out[b0 + a], y = out[b0 + L - 1 - a];
            out[b0 + a] = comp_base(y);
            out[b0 + L - 1 - a] = comp_base(x);
        }
    }
}

__global__ void __launch_bounds__(256) head_list_kernel(const unsigned long long* __restrict__ len,
                                                        const unsigned long long* __restrict__ rank,
                                                        unsigned long long n1, const unsigned long long* __restrict__ off,
                                                        unsigned long long* __restrict__ contig_off) {
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n1; i += (unsigned long long)gridDim.x * 256)
        if (len[i] || i == n1 - 1) contig_off[rank[i]] = off[i];
}

__global__ void head_flag_kernel(const unsigned long long* __restrict__ len, unsigned long long n,
                                 unsigned long long* __restrict__ flag) {
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * 256)
        flag[i] = len[i] ? 1ull : 0ull;
}

static unsigned grid_for(unsigned long long n, int num_sms) {
    unsigned long long g = (n + 255) / 256, cap = (unsigned long long)num_sms * 16;
    if (g > cap) g = cap;
    return g ? (unsigned)g : 1u;
}

constexpr unsigned kMaxRounds = 33;  // jump rounds of one ranking: log2 of the ports, plus one

// Scratch of a traversal of n survivors: links (2n u32), walks (2n u64), two
// active-port lists and the ring list (2n u32 each), two ring minima (2n u32
// each) and steps (2n u64 each), lengths, offsets, head flags and ranks
// (n + 1 u64 each), counters, scan temp.
size_t traverse_scratch_bytes(unsigned long long n) {
    return 8 * n + 16 * n + 3 * 8 * n + 2 * 8 * n + 2 * 16 * n + 4 * 8 * (n + 2) + 4 * 4 * (kMaxRounds + 2) +
           scan_temp_bytes(n + 1) + 24 * 256;
}

namespace {
struct TravBufs {
    unsigned* link;
    unsigned long long* wk;
    unsigned *act_a, *act_b, *ring;
    unsigned *ra, *rb;
    unsigned long long *sa, *sb;
    unsigned long long *len, *off, *flag, *rank;
    unsigned* cnt;  // jump rounds of the ranking, the ring count, jump rounds of the re-ranking
    void* temp;
};

TravBufs carve_traverse(void* scratch, unsigned long long n) {
    unsigned char* p = static_cast<unsigned char*>(scratch);
    auto carve = [&](size_t bytes) {
        unsigned char* r = p;
        p += (bytes + 255) & ~size_t(255);
        return r;
    };
    TravBufs t;
    t.link = reinterpret_cast<unsigned*>(carve(8 * n));
    t.wk = reinterpret_cast<unsigned long long*>(carve(16 * n));
    t.act_a = reinterpret_cast<unsigned*>(carve(8 * n));
    t.act_b = reinterpret_cast<unsigned*>(carve(8 * n));
    t.ring = reinterpret_cast<unsigned*>(carve(8 * n));
    t.ra = reinterpret_cast<unsigned*>(carve(8 * n));
    t.rb = reinterpret_cast<unsigned*>(carve(8 * n));
    t.sa = reinterpret_cast<unsigned long long*>(carve(16 * n));
    t.sb = reinterpret_cast<unsigned long long*>(carve(16 * n));
    t.len = reinterpret_cast<unsigned long long*>(carve(8 * (n + 2)));  // a scan also writes its total past the end
    t.off = reinterpret_cast<unsigned long long*>(carve(8 * (n + 2)));  // a scan also writes its total past the end
    t.flag = reinterpret_cast<unsigned long long*>(carve(8 * (n + 2)));  // a scan also writes its total past the end
    t.rank = reinterpret_cast<unsigned long long*>(carve(8 * (n + 2)));  // a scan also writes its total past the end
    t.cnt = reinterpret_cast<unsigned*>(carve(4 * 4 * (kMaxRounds + 2)));  // three runs of counters, an error count
    t.temp = carve(scan_temp_bytes(n + 1));
    return t;
}

unsigned rounds_for(unsigned long long n) {
    unsigned r = 1;
    while ((1ull << r) <= n && r < 31) ++r;
    return r;
}

// rounds + 1 jump rounds over the list act / cnt[0], in place in wk; later
// rounds find an empty list and return at once.
void jump_rounds(TravBufs& t, unsigned long long* walks, unsigned* cnt, unsigned rounds, unsigned cap_dist,
                 int num_sms, cudaStream_t s) {
    unsigned *in = t.act_a, *out = t.act_b;
    const unsigned g = (unsigned)num_sms * 16;
    for (unsigned r = 0; r <= rounds; ++r) {
        walk_jump_kernel<<<g, 256, 0, s>>>(walks, in, cnt + r, cap_dist, out, cnt + r + 1);
        std::swap(in, out);
    }
}
}  // namespace

cudaError_t launch_traverse_plan(unsigned W, const unsigned long long* keys, const unsigned char* cls,
                                 unsigned long long n, unsigned k, const unsigned* idx, unsigned long long cap,
                                 void* scratch, unsigned long long* totals, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(totals, 0, 16, s);
    if (n >= 0x7FFFFFFFull) return cudaErrorInvalidValue;  // port codes are 32-bit
    TravBufs t = carve_traverse(scratch, n);
    const unsigned long long ports = 2 * n;
    const unsigned g = grid_for(n, num_sms), gp = grid_for(ports, num_sms);
    const unsigned rounds = rounds_for(ports);
    const unsigned cap_dist = 1u << rounds;  // a walk this long has gone round a ring
    unsigned* cnt_rank = t.cnt;
    unsigned* ring_n = t.cnt + (kMaxRounds + 2);
    unsigned* cnt_rerank = t.cnt + 2 * (kMaxRounds + 2);
    unsigned* walk_err = t.cnt + 3 * (kMaxRounds + 2);
    cudaError_t e = cudaMemsetAsync(t.cnt, 0, 4 * 4 * (kMaxRounds + 2), s);
    if (e != cudaSuccess) return e;
    switch (W) {
        case 1: links_kernel<1><<<g, 256, 0, s>>>(keys, cls, n, k, idx, cap, t.link); break;
        case 2: links_kernel<2><<<g, 256, 0, s>>>(keys, cls, n, k, idx, cap, t.link); break;
        case 3: links_kernel<3><<<g, 256, 0, s>>>(keys, cls, n, k, idx, cap, t.link); break;
        case 4: links_kernel<4><<<g, 256, 0, s>>>(keys, cls, n, k, idx, cap, t.link); break;
        default: return cudaErrorInvalidValue;
    }
    // list ranking of every port by a ruling set (owners and distances in
    // ra / rb, the rulers' walks in sa: all free until the rings are found)
    e = cudaMemsetAsync(t.ra, 0xFF, 4 * ports, s);
    if (e != cudaSuccess) return e;
    ruler_walk_kernel<<<gp, 256, 0, s>>>(t.link, ports, t.ra, t.rb, t.sa, t.act_a, cnt_rank, walk_err);
    jump_rounds(t, t.sa, cnt_rank, rounds, cap_dist, num_sms, s);
    ruler_final_kernel<<<gp, 256, 0, s>>>(t.link, ports, t.ra, t.rb, t.sa, cap_dist, t.wk);
    // rings: the smallest vertex of each, cut before it, and their ports ranked again
    ring_init_kernel<<<gp, 256, 0, s>>>(t.wk, ports, cap_dist, t.link, t.ra, t.sa, t.ring, ring_n);
    unsigned n_ring = 0, n_err = 0;
    e = cudaMemcpyAsync(&n_ring, ring_n, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n_err, walk_err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (n_err) return cudaErrorUnknown;  // links that are not mutual: cannot happen
    if (n_ring) {
        const unsigned gr = grid_for(n_ring, num_sms), rr = rounds_for(n_ring);
        for (unsigned r = 0; r <= rr; ++r) {
            switch (W) {
                case 1: ring_double_kernel<1><<<gr, 256, 0, s>>>(t.ra, t.sa, t.ring, ring_n, keys, t.rb, t.sb); break;
                case 2: ring_double_kernel<2><<<gr, 256, 0, s>>>(t.ra, t.sa, t.ring, ring_n, keys, t.rb, t.sb); break;
                case 3: ring_double_kernel<3><<<gr, 256, 0, s>>>(t.ra, t.sa, t.ring, ring_n, keys, t.rb, t.sb); break;
                case 4: ring_double_kernel<4><<<gr, 256, 0, s>>>(t.ra, t.sa, t.ring, ring_n, keys, t.rb, t.sb); break;
            }
            std::swap(t.ra, t.rb);
            std::swap(t.sa, t.sb);
        }
        ring_cut_kernel<<<gr, 256, 0, s>>>(t.ra, t.ring, ring_n, t.link);
        walk_reinit_kernel<<<gr, 256, 0, s>>>(t.link, t.ring, ring_n, t.wk, t.act_a, cnt_rerank);
        jump_rounds(t, t.wk, cnt_rerank, rr, cap_dist, num_sms, s);
    }
    e = cudaMemsetAsync(t.len + n, 0, 8, s);
    if (e != cudaSuccess) return e;
    chain_len_kernel<<<g, 256, 0, s>>>(t.wk, cls, n, k, t.len);
    e = exclusive_scan_u64(t.len, t.off, n + 1, t.temp, s);  // off[n] = total bases
    if (e != cudaSuccess) return e;
    head_flag_kernel<<<grid_for(n + 1, num_sms), 256, 0, s>>>(t.len, n + 1, t.flag);
    e = exclusive_scan_u64(t.flag, t.rank, n + 1, t.temp, s);  // rank[n] = contigs
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(totals, t.off + n, 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(totals + 1, t.rank + n, 8, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_traverse_write(unsigned W, const unsigned long long* keys, const unsigned char* cls,
                                  unsigned long long n, unsigned k, unsigned long long n_contigs, void* scratch,
                                  char* out, unsigned long long* contig_off, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(contig_off, 0, 8, s);
    TravBufs t = carve_traverse(scratch, n);
    const unsigned g = grid_for(n + 1, num_sms);
    head_list_kernel<<<g, 256, 0, s>>>(t.len, t.rank, n + 1, t.off, contig_off);
    switch (W) {
        case 1: chain_write_kernel<1><<<g, 256, 0, s>>>(t.wk, cls, keys, n, k, t.off, out); break;
        case 2: chain_write_kernel<2><<<g, 256, 0, s>>>(t.wk, cls, keys, n, k, t.off, out); break;
        case 3: chain_write_kernel<3><<<g, 256, 0, s>>>(t.wk, cls, keys, n, k, t.off, out); break;
        case 4: chain_write_kernel<4><<<g, 256, 0, s>>>(t.wk, cls, keys, n, k, t.off, out); break;
        default: return cudaErrorInvalidValue;
    }
    if (n_contigs == 0) return cudaGetLastError();
    // canonical contigs: work items of kCanonChunk first-half positions
    // (chunk counts in flag, their starts in rank, first differences in sa)
    const unsigned gc = grid_for(n_contigs, num_sms);
    canon_chunks_kernel<<<gc, 256, 0, s>>>(contig_off, n_contigs, t.flag, t.sa);
    cudaError_t e = cudaMemsetAsync(t.flag + n_contigs, 0, 8, s);
    if (e == cudaSuccess) e = exclusive_scan_u64(t.flag, t.rank, n_contigs + 1, t.temp, s);
    if (e != cudaSuccess) return e;
    unsigned long long items = 0;
    e = cudaMemcpyAsync(&items, t.rank + n_contigs, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const unsigned gi = grid_for(items, num_sms);
    canon_diff_kernel<<<gi, 256, 0, s>>>(contig_off, t.rank, n_contigs, items, out, t.sa);
    canon_decide_kernel<<<gc, 256, 0, s>>>(contig_off, n_contigs, out, t.sa);
    canon_flip_kernel<<<gi, 256, 0, s>>>(contig_off, t.rank, n_contigs, items, t.sa, out);
    return cudaGetLastError();
}

}  // namespace kmer
