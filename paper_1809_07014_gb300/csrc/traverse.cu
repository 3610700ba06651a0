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
//  2. list ranking: pointer doubling over ports gives, for every port, the end
//     reached by walking out of it and the number of steps, in log2(n) rounds;
//  3. rings (ports whose walk never ends) are cut before their smallest
//     canonical k-mer (found by doubling a running minimum around the ring),
//     and the ranking is run again;
//  4. every chain is written from its end with the smaller index: the end's
//     k-mer, then one base per later vertex at its distance from the end; the
//     chains' lengths are scanned into offsets;
//  5. every contig is turned into the smaller of itself and its reverse
//     complement.
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

// Walk state of a port P: after dist steps out of P the walk stands at
// port-code `at` (a vertex and the port it would leave by next); dist 0 = P
// has no partner (the walk ends at once).
struct Walk {
    unsigned at, dist;
};

__global__ void __launch_bounds__(256) walk_init_kernel(const unsigned* __restrict__ link, unsigned long long ports,
                                                        Walk* __restrict__ wk) {
    for (unsigned long long P = blockIdx.x * 256ull + threadIdx.x; P < ports; P += (unsigned long long)gridDim.x * 256) {
        const unsigned L = link[P];
        // arriving at the partner port, the walk leaves its vertex by the other port
        wk[P] = L == kNoPort ? Walk{(unsigned)P, 0u} : Walk{L ^ 1u, 1u};
    }
}

// One round of pointer doubling: follow the walk from where it stands.
__global__ void __launch_bounds__(256) walk_double_kernel(const Walk* __restrict__ in, unsigned long long ports,
                                                          unsigned cap_dist, Walk* __restrict__ out) {
    for (unsigned long long P = blockIdx.x * 256ull + threadIdx.x; P < ports; P += (unsigned long long)gridDim.x * 256) {
        Walk w = in[P];
        if (w.dist) {
            const Walk f = in[w.at];
            if (f.dist) {
                const unsigned long long d = (unsigned long long)w.dist + f.dist;
                w.at = f.at;
                w.dist = d > cap_dist ? cap_dist : (unsigned)d;
            }
        }
        out[P] = w;
    }
}

// Rings: per port P of a ring vertex, the smallest vertex (by key) among the
// 2^r vertices met walking out of P, and where that walk stands; doubled like
// the walks.  Once 2^r passes a ring's length every port of it holds the
// ring's smallest vertex.  Ports of chain vertices keep kNoPort.
__global__ void __launch_bounds__(256) ring_init_kernel(const Walk* __restrict__ wk, unsigned long long ports,
                                                        unsigned cap_dist, const unsigned* __restrict__ link,
                                                        unsigned* __restrict__ rmin, Walk* __restrict__ step) {
    for (unsigned long long P = blockIdx.x * 256ull + threadIdx.x; P < ports; P += (unsigned long long)gridDim.x * 256) {
        const bool ring = wk[P].dist >= cap_dist;
        rmin[P] = ring ? (unsigned)(P >> 1) : kNoPort;
        step[P] = ring ? Walk{link[P] ^ 1u, 1u} : Walk{kNoPort, 0u};
    }
}

template <int W>
__global__ void __launch_bounds__(256) ring_double_kernel(const unsigned* __restrict__ rmin_in,
                                                          const Walk* __restrict__ step_in, unsigned long long ports,
                                                          const unsigned long long* __restrict__ keys,
                                                          unsigned* __restrict__ rmin_out, Walk* __restrict__ step_out) {
    for (unsigned long long P = blockIdx.x * 256ull + threadIdx.x; P < ports; P += (unsigned long long)gridDim.x * 256) {
        unsigned m = rmin_in[P];
        Walk s = step_in[P];
        if (m != kNoPort) {
            const unsigned mv = rmin_in[s.at];  // the next 2^r vertices, from where the walk stands
            unsigned long long a[W], b[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                a[w] = keys[(unsigned long long)m * W + w];
                b[w] = keys[(unsigned long long)mv * W + w];
            }
            if (key_less<W>(b, a)) m = mv;
            s = Walk{step_in[s.at].at, 0u};
        }
        rmin_out[P] = m;
        step_out[P] = s;
    }
}

// Cut every ring before its smallest vertex: drop the link of that vertex's
// port 0 and its partner's.
__global__ void __launch_bounds__(256) ring_cut_kernel(const unsigned* __restrict__ rmin, unsigned long long n,
                                                       unsigned* __restrict__ link) {
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * 256) {
        if (rmin[2 * i + 1] != (unsigned)i) continue;
        const unsigned L = link[2 * i];
        if (L != kNoPort) link[L] = kNoPort;
        link[2 * i] = kNoPort;
    }
}

// Chain of vertex i: its two ends, distances, head (the end with the smaller
// index) and i's place.  len[i] = bases of i's contig if i is a head, else 0.
__device__ __forceinline__ void chain_of(const Walk* wk, unsigned i, unsigned& head, unsigned& pos, bool& fwd,
                                         unsigned& m) {
    const Walk a = wk[2 * i], b = wk[2 * i + 1];
    const unsigned h0 = a.dist ? a.at >> 1 : i, h1 = b.dist ? b.at >> 1 : i;
    m = a.dist + b.dist + 1;
    if (h0 <= h1) {  // walking from the head reaches i through its port 0: i read as stored
        head = h0;
        pos = a.dist;
        fwd = true;
    } else {
        head = h1;
        pos = b.dist;
        fwd = false;
    }
}

__global__ void __launch_bounds__(256) chain_len_kernel(const Walk* __restrict__ wk, const unsigned char* __restrict__ cls,
                                                        unsigned long long n, unsigned k,
                                                        unsigned long long* __restrict__ len) {
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
__global__ void __launch_bounds__(256) chain_write_kernel(const Walk* __restrict__ wk,
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
            const bool stored = m == 1 || wk[2 * i + 1].dist > 0;
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

// Each contig becomes the smaller of itself and its reverse complement.
__global__ void __launch_bounds__(256) canon_contig_kernel(const unsigned long long* __restrict__ len,
                                                           const unsigned long long* __restrict__ off,
                                                           unsigned long long n, char* __restrict__ out) {
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * 256) {
        const unsigned long long L = len[i];
        if (!L) continue;
        char* c = out + off[i];
        int cmp = 0;  // sign of rc(c) - c at the first difference
        for (unsigned long long a = 0; a < L && !cmp; ++a) {
            const char r = comp_base(c[L - 1 - a]);
            if (r != c[a]) cmp = r < c[a] ? -1 : 1;
        }
        if (cmp >= 0) continue;
        for (unsigned long long a = 0, b = L - 1; a <= b && b < L; ++a, --b) {
            const char ca = c[a], cb = c[b];
            c[a] = comp_base(cb);
            c[b] = comp_base(ca);
            if (b == 0) break;
        }
    }
}

// contig_off[c] = first base of contig c (heads in vertex order), and the
// total after the last (entry n of the n + 1 scanned entries).
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

// Scratch of a traversal of n survivors: links (2n u32), two walk buffers
// (2n each), two ring minima and step buffers (2n each), and lengths,
// offsets, head flags and ranks (n + 1 u64 each), scan temp.
size_t traverse_scratch_bytes(unsigned long long n) {
    return 8 * n + 2 * 16 * n + 2 * (8 * n + 16 * n) + 4 * 8 * (n + 2) + scan_temp_bytes(n + 1) + 16 * 256;
}

namespace {
struct TravBufs {
    unsigned* link;
    Walk *wa, *wb, *sa, *sb;
    unsigned *ra, *rb;
    unsigned long long *len, *off, *flag, *rank;
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
    t.wa = reinterpret_cast<Walk*>(carve(16 * n));
    t.wb = reinterpret_cast<Walk*>(carve(16 * n));
    t.ra = reinterpret_cast<unsigned*>(carve(8 * n));
    t.rb = reinterpret_cast<unsigned*>(carve(8 * n));
    t.sa = reinterpret_cast<Walk*>(carve(16 * n));
    t.sb = reinterpret_cast<Walk*>(carve(16 * n));
    t.len = reinterpret_cast<unsigned long long*>(carve(8 * (n + 1)));
    t.off = reinterpret_cast<unsigned long long*>(carve(8 * (n + 1)));
    t.flag = reinterpret_cast<unsigned long long*>(carve(8 * (n + 1)));
    t.rank = reinterpret_cast<unsigned long long*>(carve(8 * (n + 1)));
    t.temp = carve(scan_temp_bytes(n + 1));
    return t;
}

unsigned rounds_for(unsigned long long n) {
    unsigned r = 1;
    while ((1ull << r) <= n && r < 31) ++r;
    return r;
}
}  // namespace

cudaError_t launch_traverse_plan(unsigned W, const unsigned long long* keys, const unsigned char* cls,
                                 unsigned long long n, unsigned k, const unsigned* idx, unsigned long long cap,
                                 void* scratch, unsigned long long* totals, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(totals, 0, 16, s);
    TravBufs t = carve_traverse(scratch, n);
    const unsigned long long ports = 2 * n;
    const unsigned g = grid_for(n, num_sms), gp = grid_for(ports, num_sms);
    const unsigned rounds = rounds_for(n);
    const unsigned cap_dist = 1u << rounds;  // a walk this long has gone round a ring
    switch (W) {
        case 1: links_kernel<1><<<g, 256, 0, s>>>(keys, cls, n, k, idx, cap, t.link); break;
        case 2: links_kernel<2><<<g, 256, 0, s>>>(keys, cls, n, k, idx, cap, t.link); break;
        case 3: links_kernel<3><<<g, 256, 0, s>>>(keys, cls, n, k, idx, cap, t.link); break;
        case 4: links_kernel<4><<<g, 256, 0, s>>>(keys, cls, n, k, idx, cap, t.link); break;
        default: return cudaErrorInvalidValue;
    }
    // list ranking; the final walks are left in t.wa
    auto rank_walks = [&]() {
        walk_init_kernel<<<gp, 256, 0, s>>>(t.link, ports, t.wa);
        for (unsigned r = 0; r <= rounds; ++r) {
            walk_double_kernel<<<gp, 256, 0, s>>>(t.wa, ports, cap_dist, t.wb);
            std::swap(t.wa, t.wb);
        }
    };
    rank_walks();
    // rings: the smallest vertex of each, cut before it, and the ranking again
    ring_init_kernel<<<gp, 256, 0, s>>>(t.wa, ports, cap_dist, t.link, t.ra, t.sa);
    for (unsigned r = 0; r <= rounds; ++r) {
        switch (W) {
            case 1: ring_double_kernel<1><<<gp, 256, 0, s>>>(t.ra, t.sa, ports, keys, t.rb, t.sb); break;
            case 2: ring_double_kernel<2><<<gp, 256, 0, s>>>(t.ra, t.sa, ports, keys, t.rb, t.sb); break;
            case 3: ring_double_kernel<3><<<gp, 256, 0, s>>>(t.ra, t.sa, ports, keys, t.rb, t.sb); break;
            case 4: ring_double_kernel<4><<<gp, 256, 0, s>>>(t.ra, t.sa, ports, keys, t.rb, t.sb); break;
        }
        std::swap(t.ra, t.rb);
        std::swap(t.sa, t.sb);
    }
    ring_cut_kernel<<<g, 256, 0, s>>>(t.ra, n, t.link);
    rank_walks();
    cudaError_t e = cudaMemsetAsync(t.len + n, 0, 8, s);
    if (e != cudaSuccess) return e;
    chain_len_kernel<<<g, 256, 0, s>>>(t.wa, cls, n, k, t.len);
    e = exclusive_scan_u64(t.len, t.off, n + 1, t.temp, s);  // off[n] = total bases
    if (e != cudaSuccess) return e;
    head_flag_kernel<<<grid_for(n + 1, num_sms), 256, 0, s>>>(t.len, n + 1, t.flag);
    e = exclusive_scan_u64(t.flag, t.rank, n + 1, t.temp, s);  // rank[n] = contigs
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(totals, t.off + n, 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(totals + 1, t.rank + n, 8, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    // the walks the writer reads: rank_walks ran an odd or even number of
    // doublings; keep them where the writer finds them (wa of a fresh carve)
    if (t.wa != carve_traverse(scratch, n).wa)
        e = cudaMemcpyAsync(carve_traverse(scratch, n).wa, t.wa, 16 * n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_traverse_write(unsigned W, const unsigned long long* keys, const unsigned char* cls,
                                  unsigned long long n, unsigned k, void* scratch, char* out,
                                  unsigned long long* contig_off, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(contig_off, 0, 8, s);
    TravBufs t = carve_traverse(scratch, n);
    const unsigned g = grid_for(n + 1, num_sms);
    head_list_kernel<<<g, 256, 0, s>>>(t.len, t.rank, n + 1, t.off, contig_off);
    switch (W) {
        case 1: chain_write_kernel<1><<<g, 256, 0, s>>>(t.wa, cls, keys, n, k, t.off, out); break;
        case 2: chain_write_kernel<2><<<g, 256, 0, s>>>(t.wa, cls, keys, n, k, t.off, out); break;
        case 3: chain_write_kernel<3><<<g, 256, 0, s>>>(t.wa, cls, keys, n, k, t.off, out); break;
        case 4: chain_write_kernel<4><<<g, 256, 0, s>>>(t.wa, cls, keys, n, k, t.off, out); break;
        default: return cudaErrorInvalidValue;
    }
    canon_contig_kernel<<<g, 256, 0, s>>>(t.len, t.off, n, out);
    return cudaGetLastError();
}

}  // namespace kmer
