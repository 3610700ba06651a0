/*
 * CPU oracle for k-mer analysis.  TEST INFRASTRUCTURE ONLY: the tests, the
 * package smoke check and the benchmark's CPU-baseline leg may call it; the
 * library never does.  It shares no code with the CUDA path.
 *
 * What it computes is the plain definition, written out with strings and an
 * ordered map (slow on purpose, easy to check by eye):
 *
 *  - Sec. II-B (K-mer Analysis using Distributed Histograms): every read is
 *    split into k-mers that overlap by k-1 bases; each k-mer gets a count, and
 *    the bases just before and just after it in the read are tallied as its
 *    left and right extensions.  K-mers seen fewer than min_count times are
 *    dropped (the paper keeps those "occurring more than epsilon times", so
 *    min_count = epsilon + 1).
 *  - A k-mer and its reverse complement are the same de Bruijn vertex
 *    (Sec. II-C, DNA is double stranded), so each window is stored under the
 *    smaller (lexicographic, A<C<G<T) of the two strings; when the reverse
 *    complement is kept, the two extensions swap sides and are complemented.
 *  - A window containing any byte other than A, C, G, T is skipped.  An
 *    extension base counts only if it exists in the read, is one of A/C/G/T
 *    and its Phred quality is at least qual_threshold.
 *  - Classification of each side (Sec. II-C):
 *      mode 0, depth adaptive: with m the most common extension and alt the
 *        sum of the other three tallies, the side is UNIQUE(m) iff
 *        alt <= t_hq = max(t_base, e * d) where d is the k-mer count and
 *        e = err_num / err_den (compared exactly in integers); no extension
 *        at all is DEAD_END; a tie for most common, or too many
 *        alternatives, is FORK.
 *      mode 1, static: a base is a high quality extension iff its tally is
 *        at least t_ext (Sec. II-B); exactly one such base is UNIQUE, none
 *        is DEAD_END, several are FORK.
 *    Codes 0..3 = A,C,G,T (unique), 4 = FORK, 5 = DEAD_END.
 *
 * Sharded mode (n_shards > 1) keeps only keys whose FNV-1a 64-bit hash of the
 * key string is congruent to `shard`; it is the same definition restricted to
 * a subset of keys, so that large inputs fit in host memory.  The threaded
 * form (oracle_kmer_analysis_threads) keeps a range of shards, splits the
 * reads into contiguous ranges counted by separate threads into maps of
 * their own, and adds the maps together before filtering: the counts and
 * tallies are sums over windows, and update-only inserts commute
 * (Sec. II-A, use case 1).
 */
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <queue>
#include <set>
#include <string>
#include <thread>
#include <vector>

extern "C" {

typedef struct {
    uint32_t k;
    uint32_t min_count;
    int32_t qual_offset;
    int32_t qual_threshold;
    int32_t ext_mode;
    uint32_t t_base;
    uint32_t err_num;
    uint32_t err_den;
    uint32_t t_ext;
} oracle_params;

typedef struct {
    uint64_t n;        /* surviving k-mers */
    char *keys;        /* n * k characters, ascending */
    uint64_t *count;   /* n */
    uint64_t *ext;     /* n * 8: left A,C,G,T then right A,C,G,T */
    uint8_t *cls;      /* n * 2: left, right */
    uint64_t windows;  /* valid windows counted (in this shard) */
    uint64_t distinct; /* distinct canonical k-mers before the count filter */
} oracle_result;

void oracle_free(oracle_result *r);
int oracle_kmer_analysis(const char *bases, const uint8_t *quals, const uint64_t *offsets, uint64_t n_reads,
                         const oracle_params *p, uint32_t shard, uint32_t n_shards, oracle_result *out);

}  // extern "C"

namespace {

struct Rec {
    uint64_t count = 0;
    uint64_t ext[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
};

int base_index(char c) {
    switch (c) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
    }
    return -1;
}

char complement(char c) {
    switch (c) {
        case 'A': return 'T';
        case 'C': return 'G';
        case 'G': return 'C';
        case 'T': return 'A';
    }
    return 'N';
}

std::string reverse_complement(const std::string &s) {
    std::string r(s.size(), 'N');
    for (size_t i = 0; i < s.size(); ++i) r[s.size() - 1 - i] = complement(s[i]);
    return r;
}

uint64_t fnv1a(const std::string &s) {
    uint64_t h = 14695981039346656037ull;  // FNV-1a 64 offset basis
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

const uint8_t FORK = 4, DEAD_END = 5;

uint8_t classify(const uint64_t n[4], uint64_t d, const oracle_params &p) {
    if (p.ext_mode == 1) {
        int hq = 0, which = 0;
        for (int b = 0; b < 4; ++b)
            if (n[b] >= p.t_ext) { ++hq; which = b; }
        if (hq == 0) return DEAD_END;
        if (hq == 1) return (uint8_t)which;
        return FORK;
    }
    uint64_t best = 0;
    int m = 0, ties = 0;
    for (int b = 0; b < 4; ++b) {
        if (n[b] > best) { best = n[b]; m = b; ties = 1; }
        else if (n[b] == best && best > 0) ++ties;
    }
    if (best == 0) return DEAD_END;
    if (ties > 1) return FORK;
    uint64_t alt = 0;
    for (int b = 0; b < 4; ++b)
        if (b != m) alt += n[b];
    // alt <= max(t_base, (num/den) * d)  <=>  alt*den <= max(t_base*den, num*d)
    uint64_t lhs = alt * (uint64_t)p.err_den;
    uint64_t a = (uint64_t)p.t_base * p.err_den, b = (uint64_t)p.err_num * d;
    return lhs <= (a > b ? a : b) ? (uint8_t)m : FORK;
}

// Walk every window of one read; for each window without N call
// visit(canonical key, left base/quality/exists, right base/quality/exists)
// with the extensions already in the key's orientation.
template <class Visit>
void walk_read(const std::string &read, const uint8_t *q, size_t k, const oracle_params &p, Visit visit) {
    const size_t L = read.size();
    for (size_t i = 0; i + k <= L; ++i) {
        std::string w = read.substr(i, k);
        bool ok = true;
        for (char c : w)
            if (base_index(c) < 0) ok = false;
        if (!ok) continue;
        std::string u = reverse_complement(w);
        bool flip = u < w;
        // candidate extensions in read orientation
        bool has_l = i > 0, has_r = i + k < L;
        char lb = has_l ? read[i - 1] : 'N', rb = has_r ? read[i + k] : 'N';
        int lq = has_l ? (int)q[i - 1] - p.qual_offset : -1;
        int rq = has_r ? (int)q[i + k] - p.qual_offset : -1;
        if (flip) {  // the stored key reads the other strand
            char nl = complement(rb), nr = complement(lb);
            int nlq = rq, nrq = lq;
            bool nhl = has_r, nhr = has_l;
            lb = nl; rb = nr; lq = nlq; rq = nrq; has_l = nhl; has_r = nhr;
        }
        visit(flip ? u : w, has_l && base_index(lb) >= 0 && lq >= p.qual_threshold ? base_index(lb) : -1,
              has_r && base_index(rb) >= 0 && rq >= p.qual_threshold ? base_index(rb) : -1);
    }
}

void add_window(Rec &rec, int left, int right) {
    rec.count += 1;
    if (left >= 0) rec.ext[0][left] += 1;
    if (right >= 0) rec.ext[1][right] += 1;
}

using Entry = std::pair<const std::string, Rec>;

// Keys seen at least min_count times, from `all` (every distinct key,
// ascending), with their counts, tallies and classes.
int write_result(const std::vector<const Entry *> &all, uint64_t windows, const oracle_params &p,
                 oracle_result *out) {
    const size_t k = p.k;
    std::vector<const Entry *> keep;
    for (const Entry *kv : all)
        if (kv->second.count >= p.min_count) keep.push_back(kv);
    const uint64_t n = keep.size();
    out->n = n;
    out->windows = windows;
    out->distinct = all.size();
    out->keys = (char *)std::malloc(n * k + 1);
    out->count = (uint64_t *)std::malloc(sizeof(uint64_t) * (n + 1));
    out->ext = (uint64_t *)std::malloc(sizeof(uint64_t) * (8 * n + 1));
    out->cls = (uint8_t *)std::malloc(2 * n + 1);
    if (!out->keys || !out->count || !out->ext || !out->cls) return -2;
    for (uint64_t j = 0; j < n; ++j) {
        const std::string &key = keep[j]->first;
        const Rec &rec = keep[j]->second;
        std::memcpy(out->keys + j * k, key.data(), k);
        out->count[j] = rec.count;
        for (int s = 0; s < 2; ++s)
            for (int b = 0; b < 4; ++b) out->ext[8 * j + 4 * s + b] = rec.ext[s][b];
        out->cls[2 * j + 0] = classify(rec.ext[0], rec.count, p);
        out->cls[2 * j + 1] = classify(rec.ext[1], rec.count, p);
    }
    return 0;
}

int write_result(const std::map<std::string, Rec> &M, uint64_t windows, const oracle_params &p,
                 oracle_result *out) {
    std::vector<const Entry *> all;
    all.reserve(M.size());
    for (const auto &kv : M) all.push_back(&kv);
    return write_result(all, windows, p, out);
}

}  // namespace

extern "C" int oracle_kmer_analysis(const char *bases, const uint8_t *quals, const uint64_t *offsets,
                                    uint64_t n_reads, const oracle_params *p, uint32_t shard,
                                    uint32_t n_shards, oracle_result *out) {
    if (!p || !out || (n_reads && (!bases || !quals || !offsets))) return -1;
    if (p->k == 0 || n_shards == 0 || shard >= n_shards) return -1;
    if (p->ext_mode == 0 && p->err_den == 0) return -1;
    std::memset(out, 0, sizeof(*out));
    const size_t k = p->k;
    std::map<std::string, Rec> M;
    uint64_t windows = 0;
    for (uint64_t r = 0; r < n_reads; ++r) {
        const std::string read(bases + offsets[r], bases + offsets[r + 1]);
        walk_read(read, quals + offsets[r], k, *p, [&](const std::string &c, int left, int right) {
            if (n_shards > 1 && fnv1a(c) % n_shards != shard) return;
            ++windows;
            add_window(M[c], left, right);
        });
    }
    return write_result(M, windows, *p, out);
}

/* The definition restricted to the keys whose FNV-1a hash modulo n_shards
 * lies in [shard_lo, shard_hi), with the reads split into `threads`
 * contiguous ranges counted in parallel.  Each thread fills maps of its own,
 * one per merge group (the hash divided by n_shards, modulo `threads`, so
 * that every key has one group); then thread g adds up group g's maps key by
 * key (counts and tallies are sums over windows), and the groups, disjoint
 * and each ascending, are merged into one ascending list before the count
 * filter and the classes, which see the totals. */
extern "C" int oracle_kmer_analysis_threads(const char *bases, const uint8_t *quals, const uint64_t *offsets,
                                            uint64_t n_reads, const oracle_params *p, uint32_t shard_lo,
                                            uint32_t shard_hi, uint32_t n_shards, uint32_t threads,
                                            oracle_result *out) {
    if (!p || !out || (n_reads && (!bases || !quals || !offsets))) return -1;
    if (p->k == 0 || n_shards == 0 || shard_lo >= shard_hi || shard_hi > n_shards || threads == 0) return -1;
    if (p->ext_mode == 0 && p->err_den == 0) return -1;
    std::memset(out, 0, sizeof(*out));
    const size_t k = p->k;
    const uint32_t T = threads;
    // part[t][g]: keys of merge group g seen by thread t
    std::vector<std::vector<std::map<std::string, Rec>>> part(T, std::vector<std::map<std::string, Rec>>(T));
    std::vector<uint64_t> part_windows(T, 0);
    std::vector<std::thread> pool;
    for (uint32_t t = 0; t < T; ++t) {
        const uint64_t r0 = n_reads * t / T, r1 = n_reads * (t + 1) / T;
        pool.emplace_back([&, t, r0, r1]() {
            for (uint64_t r = r0; r < r1; ++r) {
                const std::string read(bases + offsets[r], bases + offsets[r + 1]);
                walk_read(read, quals + offsets[r], k, *p, [&](const std::string &c, int left, int right) {
                    const uint64_t h = fnv1a(c);
                    const uint64_t sh = h % n_shards;
                    if (sh < shard_lo || sh >= shard_hi) return;
                    ++part_windows[t];
                    add_window(part[t][(h / n_shards) % T][c], left, right);
                });
            }
        });
    }
    for (auto &th : pool) th.join();
    pool.clear();
    std::vector<std::map<std::string, Rec>> group(T);
    for (uint32_t g = 0; g < T; ++g) {
        pool.emplace_back([&, g]() {
            for (uint32_t t = 0; t < T; ++t) {
                for (const auto &kv : part[t][g]) {
                    Rec &rec = group[g][kv.first];
                    rec.count += kv.second.count;
                    for (int s = 0; s < 2; ++s)
                        for (int b = 0; b < 4; ++b) rec.ext[s][b] += kv.second.ext[s][b];
                }
                std::map<std::string, Rec>().swap(part[t][g]);
            }
        });
    }
    for (auto &th : pool) th.join();
    uint64_t windows = 0, distinct = 0;
    for (uint32_t t = 0; t < T; ++t) windows += part_windows[t];
    for (uint32_t g = 0; g < T; ++g) distinct += group[g].size();
    // k-way merge of the groups into ascending order
    using It = std::map<std::string, Rec>::const_iterator;
    auto later = [](const std::pair<It, It> &a, const std::pair<It, It> &b) { return b.first->first < a.first->first; };
    std::priority_queue<std::pair<It, It>, std::vector<std::pair<It, It>>, decltype(later)> heads(later);
    for (uint32_t g = 0; g < T; ++g)
        if (!group[g].empty()) heads.push({group[g].cbegin(), group[g].cend()});
    std::vector<const Entry *> all;
    all.reserve(distinct);
    while (!heads.empty()) {
        auto h = heads.top();
        heads.pop();
        all.push_back(&*h.first);
        if (++h.first != h.second) heads.push(h);
    }
    return write_result(all, windows, *p, out);
}

/* Merge of Algorithm 1 (Sec. II-G): the k-mer set of the reads (the
 * definition above, with its count filter) and ExtractKmers(C, k), the
 * k-mers of the contigs C, which the paper treats as error-free k-mers with
 * unique high-quality extensions.  Reading taken here:
 *  - a contig k-mer's extension on a side is the contig's neighbouring base
 *    there (none at a contig end), in the k-mer's canonical orientation;
 *    over all its occurrences in C a side has a set of such bases: one base
 *    makes the side UNIQUE, none DEAD_END, two or more FORK (every contig base
 *    is high quality, so no count threshold applies);
 *  - a k-mer in both sets is kept once, with the reads' record;
 *  - a k-mer only in the contigs is added with count 0, zero tallies and the
 *    classes above.
 * The result is ascending by key. */
extern "C" int oracle_merge_contigs(const char *bases, const uint8_t *quals, const uint64_t *offsets,
                                    uint64_t n_reads, const oracle_params *p, const char *contigs,
                                    const uint64_t *coffsets, uint64_t n_contigs, oracle_result *out) {
    if (!p || !out || (n_contigs && (!contigs || !coffsets))) return -1;
    oracle_result reads{};
    int rc = oracle_kmer_analysis(bases, quals, offsets, n_reads, p, 0, 1, &reads);
    if (rc) {
        oracle_free(&reads);
        return rc;
    }
    const size_t k = p->k;
    // k-mers of the contigs and their neighbour sets (every contig base counts as high quality)
    oracle_params cp = *p;
    cp.qual_offset = 0;
    cp.qual_threshold = 0;
    std::map<std::string, std::set<int>[2]> ck;
    for (uint64_t c = 0; c < n_contigs; ++c) {
        const std::string contig(contigs + coffsets[c], contigs + coffsets[c + 1]);
        const std::vector<uint8_t> q(contig.size(), 0);
        walk_read(contig, q.data(), k, cp, [&](const std::string &key, int left, int right) {
            auto &sides = ck[key];
            if (left >= 0) sides[0].insert(left);
            if (right >= 0) sides[1].insert(right);
        });
    }
    // union: the reads' records, then the contig-only k-mers
    std::map<std::string, size_t> from_reads;  // key -> row of `reads`
    for (uint64_t j = 0; j < reads.n; ++j) from_reads[std::string(reads.keys + j * k, reads.keys + (j + 1) * k)] = j;
    std::vector<std::string> added;
    for (const auto &kv : ck)
        if (!from_reads.count(kv.first)) added.push_back(kv.first);
    const uint64_t n = reads.n + added.size();
    out->n = n;
    out->windows = reads.windows;
    out->distinct = reads.distinct;
    out->keys = (char *)std::malloc(n * k + 1);
    out->count = (uint64_t *)std::malloc(sizeof(uint64_t) * (n + 1));
    out->ext = (uint64_t *)std::malloc(sizeof(uint64_t) * (8 * n + 1));
    out->cls = (uint8_t *)std::malloc(2 * n + 1);
    if (!out->keys || !out->count || !out->ext || !out->cls) {
        oracle_free(&reads);
        return -2;
    }
    // ascending merge of the two sorted lists
    uint64_t i = 0, a = 0, o = 0;
    while (i < reads.n || a < added.size()) {
        const bool take_read =
            a == added.size() || (i < reads.n && std::string(reads.keys + i * k, reads.keys + (i + 1) * k) < added[a]);
        if (take_read) {
            std::memcpy(out->keys + o * k, reads.keys + i * k, k);
            out->count[o] = reads.count[i];
            for (int e = 0; e < 8; ++e) out->ext[8 * o + e] = reads.ext[8 * i + e];
            out->cls[2 * o] = reads.cls[2 * i];
            out->cls[2 * o + 1] = reads.cls[2 * i + 1];
            ++i;
        } else {
            const auto &sides = ck[added[a]];
            std::memcpy(out->keys + o * k, added[a].data(), k);
            out->count[o] = 0;
            for (int e = 0; e < 8; ++e) out->ext[8 * o + e] = 0;
            for (int s2 = 0; s2 < 2; ++s2)
                out->cls[2 * o + s2] = sides[s2].empty() ? DEAD_END
                                                         : (sides[s2].size() == 1 ? (uint8_t)*sides[s2].begin() : FORK);
            ++a;
        }
        ++o;
    }
    oracle_free(&reads);
    return 0;
}

/* De Bruijn graph traversal (Sec. II-C): contigs are the paths formed by
 * k-mers with unique extensions.  Reading taken here:
 *  - a vertex is a k-mer of the set whose two sides are both UNIQUE (classes
 *    0..3); a k-mer x read in either orientation has, in that orientation, a
 *    left base l(x) and a right base r(x) (for the reverse complement of a
 *    stored k-mer: the complements of its right and left classes);
 *  - x and y = x[1..k) + r(x) are joined when y's canonical form is a vertex
 *    other than x's and l(y) = x[0] (each names the other); a k-mer followed
 *    by its own reverse complement (a hairpin) is joined to nothing there, so
 *    that every contig uses a k-mer at most once;
 *  - a contig is a maximal path: its first k-mer, then the right base of every
 *    later k-mer; a cycle is cut before its smallest canonical k-mer and read
 *    from that k-mer in its stored orientation;
 *  - each contig is reported as the smaller of its string and its reverse
 *    complement, and the contigs in ascending order.
 * The contigs are written to *contigs (malloc'd, concatenated) with
 * *offsets (n_contigs + 1 entries, malloc'd). */
extern "C" int oracle_traverse(const char *keys, const uint8_t *cls, uint64_t n, uint32_t k, char **contigs,
                               uint64_t **offsets, uint64_t *n_contigs) {
    if ((n && (!keys || !cls)) || !contigs || !offsets || !n_contigs || k == 0) return -1;
    std::map<std::string, std::pair<int, int>> vert;  // canonical k-mer -> (left, right) of its stored orientation
    for (uint64_t i = 0; i < n; ++i)
        if (cls[2 * i] < 4 && cls[2 * i + 1] < 4) vert[std::string(keys + i * k, keys + (i + 1) * k)] = {cls[2 * i], cls[2 * i + 1]};
    const char *base = "ACGT";
    auto canon = [](const std::string &x) {
        const std::string r = reverse_complement(x);
        return r < x ? r : x;
    };
    // left and right base of x in its own orientation, or false if x is no vertex
    auto sides = [&](const std::string &x, int &l, int &r) {
        const std::string c = canon(x);
        auto it = vert.find(c);
        if (it == vert.end()) return false;
        if (c == x) {
            l = it->second.first;
            r = it->second.second;
        } else {
            l = 3 - it->second.second;
            r = 3 - it->second.first;
        }
        return true;
    };
    auto next = [&](const std::string &x, std::string &y) {  // the vertex joined to x's right, if any
        int l, r, l2, r2;
        if (!sides(x, l, r)) return false;
        y = x.substr(1) + base[r];
        return canon(y) != canon(x) && sides(y, l2, r2) && base[l2] == x[0];
    };
    auto prev = [&](const std::string &x, std::string &y) {  // the vertex joined to x's left, if any
        int l, r, l2, r2;
        if (!sides(x, l, r)) return false;
        y = std::string(1, base[l]) + x.substr(0, x.size() - 1);
        return canon(y) != canon(x) && sides(y, l2, r2) && base[r2] == x[x.size() - 1];
    };
    std::set<std::string> used;
    std::vector<std::string> out;
    for (const auto &kv : vert) {
        if (used.count(kv.first)) continue;
        // walk left to the path's start, or around a cycle back to this k-mer
        std::string x = kv.first, y;
        bool cycle = false;
        while (prev(x, y)) {
            if (canon(y) == kv.first) {
                cycle = true;
                break;
            }
            x = y;
        }
        if (cycle) {  // start at the cycle's smallest canonical k-mer, stored orientation
            std::string m = kv.first, z = kv.first;
            while (next(z, y) && canon(y) != kv.first) {
                z = y;
                if (canon(z) < m) m = canon(z);
            }
            x = m;
        }
        std::string contig = x;
        used.insert(canon(x));
        while (next(x, y) && !used.count(canon(y))) {
            contig += y.back();
            used.insert(canon(y));
            x = y;
        }
        const std::string rc = reverse_complement(contig);
        out.push_back(rc < contig ? rc : contig);
    }
    std::sort(out.begin(), out.end());
    uint64_t total = 0;
    for (const auto &c : out) total += c.size();
    *contigs = (char *)std::malloc(total + 1);
    *offsets = (uint64_t *)std::malloc(sizeof(uint64_t) * (out.size() + 1));
    if (!*contigs || !*offsets) return -2;
    (*offsets)[0] = 0;
    for (size_t i = 0; i < out.size(); ++i) {
        std::memcpy(*contigs + (*offsets)[i], out[i].data(), out[i].size());
        (*offsets)[i + 1] = (*offsets)[i] + out[i].size();
    }
    *n_contigs = out.size();
    return 0;
}

extern "C" void oracle_free_contigs(char *contigs, uint64_t *offsets) {
    std::free(contigs);
    std::free(offsets);
}

extern "C" void oracle_free(oracle_result *r) {
    if (!r) return;
    std::free(r->keys);
    std::free(r->count);
    std::free(r->ext);
    std::free(r->cls);
    std::memset(r, 0, sizeof(*r));
}

extern "C" uint64_t oracle_fnv1a(const char *s, uint64_t len) {
    return fnv1a(std::string(s, s + len));
}

/* The same definition restricted to an explicit set of canonical keys
 * (n_keys strings of k characters, each the smaller of itself and its
 * reverse complement): count[i], ext[8i..8i+8) and cls[2i..2i+2) of key i,
 * accumulated over the given reads.  Counts add across calls on disjoint
 * read ranges (update-only inserts commute, Sec. II-A use case 1), so a
 * caller may split the reads over threads and sum. */
extern "C" int oracle_count_keys(const char *bases, const uint8_t *quals, const uint64_t *offsets, uint64_t n_reads,
                                 const oracle_params *p, const char *keys, uint64_t n_keys, uint64_t *count,
                                 uint64_t *ext) {
    if (!p || (n_reads && (!bases || !quals || !offsets)) || (n_keys && (!keys || !count || !ext))) return -1;
    const size_t k = p->k;
    std::map<std::string, uint64_t> index;
    for (uint64_t i = 0; i < n_keys; ++i) index[std::string(keys + i * k, keys + (i + 1) * k)] = i;
    std::vector<Rec> recs(n_keys);
    for (uint64_t r = 0; r < n_reads; ++r) {
        const std::string read(bases + offsets[r], bases + offsets[r + 1]);
        walk_read(read, quals + offsets[r], k, *p, [&](const std::string &c, int left, int right) {
            auto it = index.find(c);
            if (it != index.end()) add_window(recs[it->second], left, right);
        });
    }
    for (uint64_t i = 0; i < n_keys; ++i) {
        count[i] += recs[i].count;
        for (int s = 0; s < 2; ++s)
            for (int b = 0; b < 4; ++b) ext[8 * i + 4 * s + b] += recs[i].ext[s][b];
    }
    return 0;
}

/* Classes of one k-mer from its summed tallies (the rule of oracle_kmer_analysis). */
extern "C" void oracle_classify(const uint64_t *ext8, uint64_t count, const oracle_params *p, uint8_t *cls2) {
    cls2[0] = classify(ext8, count, *p);
    cls2[1] = classify(ext8 + 4, count, *p);
}
