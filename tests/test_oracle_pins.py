"""Pins for the CPU oracle, independent of the oracle itself.

Each check comes from something other than the oracle's own code: a brute
force O(n^2) scan written differently, closed forms derived by hand from the
definition of k-mer analysis (Sec. II-B of the paper) and of the extension
classes (Sec. II-C), invariants of that definition (order independence of
update-only inserts, Sec. II-A use case 1; strand symmetry), and the
generator's ground truth (read placements on known genomes).
"""
import itertools
import random

import numpy as np
import pytest

import oracle
import synth
from tests import helpers

COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}
ORDER = "ACGT"


# ---------------------------------------------------------------- brute force
def brute_force(reads, p: oracle.Params):
    """Quadratic scan: a list of [key, count, ext] searched linearly per window."""
    table = []  # list of [key, count, [[4],[4]]]
    k = p.k
    for seq, qual in reads:
        seq = seq.decode() if isinstance(seq, bytes) else seq
        for i in range(len(seq) - k + 1):
            w = seq[i:i + k]
            if any(ch not in ORDER for ch in w):
                continue
            rc = "".join(COMP[ch] for ch in reversed(w))
            # (left base, left qual) and (right base, right qual) in the orientation of the key
            left = (seq[i - 1], qual[i - 1]) if i > 0 else None
            right = (seq[i + k], qual[i + k]) if i + k < len(seq) else None
            if rc < w:
                w, left, right = rc, (None if right is None else (COMP.get(right[0], "N"), right[1])), \
                    (None if left is None else (COMP.get(left[0], "N"), left[1]))
            hit = None
            for row in table:
                if row[0] == w:
                    hit = row
                    break
            if hit is None:
                hit = [w, 0, [[0] * 4, [0] * 4]]
                table.append(hit)
            hit[1] += 1
            for side, e in ((0, left), (1, right)):
                if e is not None and e[0] in ORDER and e[1] - p.qual_offset >= p.qual_threshold:
                    hit[2][side][ORDER.index(e[0])] += 1
    out = []
    for key, cnt, ext in sorted(table, key=lambda r: r[0]):
        if cnt >= p.min_count:
            out.append((key, cnt, ext[0] + ext[1], (bf_class(ext[0], cnt, p), bf_class(ext[1], cnt, p))))
    return out, sum(r[1] for r in table), len(table)


def bf_class(n, d, p):
    if p.ext_mode == 1:
        hq = [b for b in range(4) if n[b] >= p.t_ext]
        return 5 if not hq else (hq[0] if len(hq) == 1 else 4)
    if max(n) == 0:
        return 5
    for b in range(4):
        others = [n[x] for x in range(4) if x != b]
        if all(n[b] > o for o in others):
            alt = sum(others)
            return b if alt * p.err_den <= max(p.t_base * p.err_den, p.err_num * d) else 4
    return 4  # no strict maximum


def as_rows(res: oracle.Result):
    return [(res.keys[i].decode(), int(res.count[i]), [int(x) for x in res.ext[i]],
             (int(res.cls[i, 0]), int(res.cls[i, 1]))) for i in range(len(res))]


def random_reads(rng, n, lmin, lmax, alphabet="ACGT", n_rate=0.0):
    reads = []
    for _ in range(n):
        L = rng.randint(lmin, lmax)
        s = "".join(("N" if rng.random() < n_rate else rng.choice(alphabet)) for _ in range(L))
        q = bytes(33 + rng.randint(2, 41) for _ in range(L))
        reads.append((s.encode(), q))
    return reads


def test_brute_force_exhaustive_short_reads():
    """Every read over {A,C,G,T,N} of length <= 5, every k <= length."""
    for L in range(1, 6):
        for tup in itertools.product("ACGTN", repeat=L):
            s = "".join(tup).encode()
            q = bytes(33 + 20 + (i % 3) * 10 - 10 for i in range(L))  # Phred 10, 20, 30 ...
            for k in range(1, L + 1):
                p = oracle.Params(k=k, min_count=1)
                want, _, _ = brute_force([(s, q)], p)
                got = oracle.run_reads([(s, q)], p)
                assert as_rows(got) == want, (s, k)


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_random_sets(seed):
    rng = random.Random(seed)
    reads = random_reads(rng, rng.randint(1, 20), 1, 40, alphabet=rng.choice(["ACGT", "AC", "ACGT"]),
                         n_rate=rng.choice([0.0, 0.02]))
    k = rng.choice([1, 2, 3, 5, 7, 11, 13])
    p = oracle.Params(k=k, min_count=rng.choice([1, 2, 3]), qual_threshold=rng.choice([0, 20, 30]),
                      ext_mode=rng.choice([0, 1]), t_base=rng.choice([0, 1, 2]),
                      err_num=rng.choice([0, 1, 3]), err_den=rng.choice([1, 10]), t_ext=rng.choice([1, 2]))
    want, windows, distinct = brute_force(reads, p)
    got = oracle.run_reads(reads, p)
    assert as_rows(got) == want
    assert got.windows == windows and got.distinct == distinct


# -------------------------------------------------------------- closed forms
def test_homopolymer():
    """A^L: one key A^k, count L-k+1, L-k left and L-k right extensions, all A."""
    for L, k in [(10, 3), (150, 21), (150, 99), (40, 40)]:
        for base in "AT":  # T^L is the reverse complement of A^L: same vertex
            res = oracle.run_reads([(base.encode() * L, b"I" * L)], oracle.Params(k=k, min_count=1))
            assert [r[0] for r in as_rows(res)] == ["A" * k]
            assert int(res.count[0]) == L - k + 1
            assert list(res.ext[0]) == [L - k, 0, 0, 0, L - k, 0, 0, 0]
            expect = 0 if L > k else oracle.DEAD_END
            assert tuple(res.cls[0]) == (expect, expect)


def de_bruijn(k):
    """Linear de Bruijn sequence of order k over ACGT (Lyndon-word construction)."""
    a = [0] * (4 * k)
    seq = []

    def db(t, p):
        if t > k:
            if k % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            db(t + 1, p)
            for j in range(a[t - p] + 1, 4):
                a[t] = j
                db(t + 1, t)

    db(1, 1)
    s = "".join(ORDER[x] for x in seq)
    return s + s[:k - 1]


@pytest.mark.parametrize("k", [1, 3, 5, 7])
def test_de_bruijn_sequence(k):
    """Every k-mer occurs once as a window; for odd k no k-mer is its own reverse
    complement, so each canonical k-mer is counted exactly twice."""
    s = de_bruijn(k)
    assert len(s) == 4 ** k + k - 1
    res = oracle.run_reads([(s.encode(), b"I" * len(s))], oracle.Params(k=k, min_count=1))
    assert len(res) == 4 ** k // 2 == res.distinct
    assert (res.count == 2).all()
    assert res.windows == 4 ** k


def test_k_equals_read_length_has_no_extensions():
    rng = random.Random(5)
    reads = random_reads(rng, 30, 25, 25)
    res = oracle.run_reads(reads, oracle.Params(k=25, min_count=1))
    assert res.windows == 30 and (res.ext == 0).all() and (res.cls == oracle.DEAD_END).all()


def test_reads_shorter_than_k_and_all_n():
    res = oracle.run_reads([(b"ACGT", b"IIII"), (b"NNNNNNNN", b"########")], oracle.Params(k=5, min_count=1))
    assert len(res) == 0 and res.windows == 0 and res.distinct == 0
    res = oracle.run_reads([(b"ACGNACGNACGN", b"I" * 12)], oracle.Params(k=4, min_count=1))
    assert len(res) == 0 and res.windows == 0


def test_low_quality_gives_dead_ends_but_counts_windows():
    rng = random.Random(7)
    reads = [(s, bytes(33 + 19 for _ in s)) for s, _ in random_reads(rng, 20, 30, 60)]
    res = oracle.run_reads(reads, oracle.Params(k=7, min_count=1, qual_threshold=20))
    assert (res.ext == 0).all() and (res.cls == oracle.DEAD_END).all()
    assert res.windows == sum(len(s) - 6 for s, _ in reads)
    # threshold is inclusive: Phred 19 >= 19 counts
    res = oracle.run_reads(reads, oracle.Params(k=7, min_count=1, qual_threshold=19))
    assert res.ext.sum() > 0


def build_ext_case(x: str, left_counts, bare: int):
    """Reads giving k-mer x (canonical) exactly the left tallies `left_counts`
    plus `bare` occurrences with no extension on either side."""
    reads = []
    for b, n in zip(ORDER, left_counts):
        reads += [((b + x).encode(), b"I" * (len(x) + 1))] * n
    reads += [(x.encode(), b"I" * len(x))] * bare
    return reads


@pytest.mark.parametrize("left,bare,params,expect", [
    # depth adaptive, t_base = 2, e = 1/10: UNIQUE iff alt <= max(2, d/10)
    ([10, 2, 0, 0], 0, dict(t_base=2, err_num=1, err_den=10), 0),
    ([10, 3, 0, 0], 0, dict(t_base=2, err_num=1, err_den=10), 4),
    ([30, 3, 0, 0], 0, dict(t_base=2, err_num=1, err_den=10), 0),
    ([30, 4, 0, 0], 0, dict(t_base=2, err_num=1, err_den=10), 4),
    # exact boundary of e*d: alt = 3, d = 30 -> 3*10 <= 30: unique; d = 29 -> fork
    ([0, 0, 20, 3], 7, dict(t_base=1, err_num=1, err_den=10), 2),
    ([0, 0, 20, 3], 6, dict(t_base=1, err_num=1, err_den=10), 4),
    ([5, 5, 0, 0], 0, dict(t_base=100, err_num=1, err_den=1), 4),  # tie for most common
    ([0, 0, 0, 0], 9, dict(t_base=2, err_num=1, err_den=10), 5),   # no extension
    ([0, 0, 0, 1], 0, dict(t_base=0, err_num=0, err_den=1), 3),
    ([1, 0, 0, 1], 0, dict(t_base=5, err_num=0, err_den=1), 4),
])
def test_classification_depth_adaptive(left, bare, params, expect):
    x = "ACCGTTGAC"  # its reverse complement GTCAACGGT is larger, so x is the key
    assert x < "".join(COMP[c] for c in reversed(x))
    res = oracle.run_reads(build_ext_case(x, left, bare), oracle.Params(k=len(x), min_count=1, **params))
    rows = {r[0]: r for r in as_rows(res)}
    assert rows[x][1] == sum(left) + bare
    assert rows[x][2][:4] == list(left)
    assert rows[x][3][0] == expect
    assert rows[x][3][1] == 5  # nothing follows x in these reads


@pytest.mark.parametrize("left,t_ext,expect", [
    ([2, 1, 0, 0], 2, 0), ([2, 2, 0, 0], 2, 4), ([1, 1, 1, 1], 2, 5), ([0, 0, 0, 7], 7, 3), ([0, 0, 0, 6], 7, 5),
])
def test_classification_static(left, t_ext, expect):
    x = "ACCGTTGAC"
    res = oracle.run_reads(build_ext_case(x, left, 0), oracle.Params(k=len(x), min_count=1, ext_mode=1, t_ext=t_ext))
    rows = {r[0]: r for r in as_rows(res)}
    assert rows[x][3][0] == expect


def test_flipped_windows_swap_and_complement_extensions():
    """Read G+rc(x)+T: the window rc(x) is stored as x with left comp(T)=A and right comp(G)=C."""
    x = "ACCGTTGAC"
    rcx = "".join(COMP[c] for c in reversed(x))
    res = oracle.run_reads([(("G" + rcx + "T").encode(), b"I" * (len(x) + 2))], oracle.Params(k=len(x), min_count=1))
    rows = {r[0]: r for r in as_rows(res)}
    assert rows[x][2] == [1, 0, 0, 0, 0, 1, 0, 0]


# -------------------------------------------------------------- invariants
def small_metagenome(n_reads=3000, seed=11, **kw):
    r = synth.Recipe("pin", seed=seed, n_genomes=3, genome_len_min=3000, genome_len_max=6000,
                     abundance_sigma=1.0, n_reads=n_reads, read_len_min=40, read_len_max=150,
                     subst_rate=0.01, err_qual_lo=2, err_qual_hi=12, n_rate=0.002, **kw)
    return synth.generate(r)


def reads_of(rs):
    return [rs.read(i) for i in range(rs.n_reads)]


def test_invariants_on_synthetic_reads():
    rs = small_metagenome()
    reads = reads_of(rs)
    for k in (5, 21, 33):
        p1 = oracle.Params(k=k, min_count=1)
        full = oracle.run_reads(reads, p1)
        # total count = valid windows, counted by a separate scan
        valid = sum(1 for s, _ in reads for i in range(len(s) - k + 1) if b"N" not in s[i:i + k])
        assert int(full.count.sum()) == full.windows == valid
        assert full.distinct == len(full)
        # tallies never exceed the count, per side
        assert (full.ext[:, :4].sum(1) <= full.count).all() and (full.ext[:, 4:].sum(1) <= full.count).all()
        # no key contains N, every key is canonical
        for key in full.keys[:2000]:
            s = key.decode()
            assert set(s) <= set(ORDER)
            assert s <= "".join(COMP[c] for c in reversed(s))
        # reverse complementing every read (qualities reversed) changes nothing
        rc_reads = [("".join(COMP.get(c, "N") for c in reversed(s.decode())).encode(), q[::-1]) for s, q in reads]
        assert as_rows(oracle.run_reads(rc_reads, p1)) == as_rows(full)
        # read order does not matter (update-only inserts commute)
        perm = reads[:]
        random.Random(k).shuffle(perm)
        assert as_rows(oracle.run_reads(perm, p1)) == as_rows(full)
        # a higher count threshold gives exactly the subset with count >= threshold
        p3 = oracle.Params(k=k, min_count=3)
        sub = oracle.run_reads(reads, p3)
        keep = full.count >= 3
        assert list(sub.keys) == list(full.keys[keep]) and (sub.ext == full.ext[keep]).all()
        # shards partition the key set
        parts = [oracle.run(rs.bases, rs.quals, rs.offsets, p1, s, 4) for s in range(4)]
        merged = sorted(r for part in parts for r in as_rows(part))
        assert merged == as_rows(full)
        assert sum(part.windows for part in parts) == full.windows


def test_shard_hash_is_fnv1a():
    # FNV-1a 64 reference values (offset basis, prime 1099511628211)
    assert oracle.fnv1a(b"") == 0xCBF29CE484222325
    assert oracle.fnv1a(b"a") == 0xAF63DC4C8601EC8C


# ------------------------------------------------------ generator ground truth
def ground_truth_counts(rs, k):
    """Counts and extension tallies from read placements on the known genomes.

    Error-free reads are exact genome substrings (or their reverse complements),
    so the window at genome position x is covered by every read starting in
    [x - L + k, x]; its left neighbour x-1 is inside the read iff the read
    starts at or before x-1, its right neighbour x+k iff it ends after x+k.
    """
    L = int(rs.recipe.read_len_min)
    assert rs.recipe.read_len_max == L
    table = {}
    gstart = np.concatenate([[0], np.cumsum(rs.genome_lens)]).astype(np.int64)
    for g in range(len(rs.genome_lens)):
        seq = rs.genomes[gstart[g]:gstart[g + 1]].tobytes().decode()
        G = len(seq)
        starts = np.zeros(G + 1, dtype=np.int64)
        np.add.at(starts, rs.truth_pos[rs.truth_genome == g].astype(np.int64), 1)
        cum = np.concatenate([[0], np.cumsum(starts)])  # cum[j] = reads starting before j

        def reads_starting(lo, hi):  # starts in [lo, hi]
            lo, hi = max(lo, 0), min(hi, G - L)
            return 0 if hi < lo else int(cum[hi + 1] - cum[lo])

        for x in range(G - k + 1):
            cov = reads_starting(x - L + k, x)
            if cov == 0:
                continue
            w = seq[x:x + k]
            nl = reads_starting(x - L + k, x - 1)   # also contain x-1
            nr = reads_starting(x - L + k + 1, x)   # also contain x+k
            lb = seq[x - 1] if x > 0 else None
            rb = seq[x + k] if x + k < G else None
            rc = "".join(COMP[c] for c in reversed(w))
            if rc < w:
                w, lb, rb, nl, nr = rc, (COMP[rb] if rb else None), (COMP[lb] if lb else None), nr, nl
            row = table.setdefault(w, [0, [0] * 8])
            row[0] += cov
            if lb and nl:
                row[1][ORDER.index(lb)] += nl
            if rb and nr:
                row[1][4 + ORDER.index(rb)] += nr
    return table


@pytest.mark.parametrize("k", [11, 21, 31])
def test_generator_ground_truth(k):
    r = synth.Recipe("truth", seed=3, n_genomes=2, genome_len_min=4000, genome_len_max=7000,
                     abundance_sigma=0.5, n_reads=1500, read_len_min=100, read_len_max=100,
                     subst_rate=0.0, qual_min=30, qual_max=41)
    rs = synth.generate(r, truth=True)
    truth = ground_truth_counts(rs, k)
    res = oracle.run(rs.bases, rs.quals, rs.offsets, oracle.Params(k=k, min_count=1))
    got = {row[0]: [row[1], row[2]] for row in as_rows(res)}
    assert got == truth


def test_count_keys_matches_full_definition():
    """The key-set mode equals the full oracle restricted to those keys, for any
    split of the reads over threads; keys never seen get zero counts."""
    rs = small_metagenome(n_reads=2500, seed=5)
    for k in (21, 33):
        p = oracle.Params(k=k, min_count=1)
        full = oracle.run(rs.bases, rs.quals, rs.offsets, p)
        idx = np.random.default_rng(k).choice(len(full), 200, replace=False)
        for threads in (1, 3):
            c, e, cl = oracle.count_keys(rs.bases, rs.quals, rs.offsets, p, full.keys[idx], threads=threads)
            assert (c == full.count[idx]).all() and (e == full.ext[idx]).all() and (cl == full.cls[idx]).all()
        absent = np.array([b"A" * k], dtype=f"S{k}")
        if absent[0] not in set(full.keys):
            c, e, cl = oracle.count_keys(rs.bases, rs.quals, rs.offsets, p, absent, threads=2)
            assert c[0] == 0 and (e == 0).all() and tuple(cl[0]) == (oracle.DEAD_END, oracle.DEAD_END)


@pytest.mark.parametrize("seed", range(12))
def test_threaded_sharded_mode_against_brute_force(seed):
    """The threaded form (reads split over threads, partial maps summed before
    the filter) restricted to a shard range equals the brute-force scan
    restricted to the keys whose FNV-1a hash falls in that range."""
    rng = random.Random(1000 + seed)
    reads = random_reads(rng, rng.randint(1, 30), 1, 40, alphabet=rng.choice(["ACGT", "AC"]),
                         n_rate=rng.choice([0.0, 0.03]))
    k = rng.choice([1, 3, 5, 7, 11])
    p = oracle.Params(k=k, min_count=rng.choice([1, 2, 3]), qual_threshold=rng.choice([0, 20, 30]),
                      ext_mode=rng.choice([0, 1]))
    bases = b"".join(r[0] for r in reads)
    quals = b"".join(r[1] for r in reads)
    offsets = np.zeros(len(reads) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([len(r[0]) for r in reads], dtype=np.uint64)
    full, _, _ = brute_force(reads, p)
    n_shards = rng.choice([1, 2, 5])
    lo = rng.randrange(n_shards)
    hi = rng.randrange(lo + 1, n_shards + 1)
    want = [row for row in full if lo <= helpers.fnv1a_keys(np.array([row[0]], dtype=f"S{k}"))[0] % n_shards < hi]
    for threads in (1, 2, 3, 7):
        got = oracle.run_threads(bases, quals, offsets, p, lo, hi, n_shards, threads)
        assert as_rows(got) == want, (threads, lo, hi, n_shards)


def test_threaded_mode_equals_single_thread_on_a_metagenome_slice():
    rs = synth.generate(synth.METAGENOME_2G.scaled(3000))
    p = oracle.Params(k=31)
    one = oracle.run(rs.bases, rs.quals, rs.offsets, p)
    many = oracle.run_threads(rs.bases, rs.quals, rs.offsets, p, threads=5)
    assert as_rows(many) == as_rows(one)
    assert (many.windows, many.distinct) == (one.windows, one.distinct)
    parts = [oracle.run_threads(rs.bases, rs.quals, rs.offsets, p, lo, lo + 3, 9, threads=4) for lo in (0, 3, 6)]
    assert sum(x.windows for x in parts) == one.windows
    assert sum(x.distinct for x in parts) == one.distinct
    merged = sorted(r for x in parts for r in as_rows(x))
    assert merged == as_rows(one)


# ------------------------------------------------------ merge with contig k-mers
def contig_kmers_brute(contigs, k):
    """ExtractKmers of Algorithm 1, written out: canonical k-mer -> the sets of
    its left and right neighbours over all occurrences in the contigs."""
    table = {}
    for c in contigs:
        c = c.decode() if isinstance(c, bytes) else c
        for i in range(len(c) - k + 1):
            w = c[i:i + k]
            if any(ch not in ORDER for ch in w):
                continue
            left = c[i - 1] if i > 0 else None
            right = c[i + k] if i + k < len(c) else None
            rc = "".join(COMP[ch] for ch in reversed(w))
            if rc < w:
                w, left, right = rc, (COMP.get(right) if right else None), (COMP.get(left) if left else None)
            sides = table.setdefault(w, (set(), set()))
            if left is not None and left in ORDER:
                sides[0].add(left)
            if right is not None and right in ORDER:
                sides[1].add(right)
    return table


def merge_brute(reads, contigs, p):
    rows, _, _ = brute_force(reads, p)
    have = {r[0] for r in rows}
    out = list(rows)
    for key, (ls, rs) in contig_kmers_brute(contigs, p.k).items():
        if key in have:
            continue
        cl = tuple(5 if not s else (ORDER.index(next(iter(s))) if len(s) == 1 else 4) for s in (ls, rs))
        out.append((key, 0, [0] * 8, cl))
    return sorted(out, key=lambda r: r[0])


def flat(seqs):
    data = b"".join(seqs)
    offs = np.zeros(len(seqs) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(x) for x in seqs], dtype=np.uint64)
    return data, offs


def test_merge_hand_case():
    """Reads ACGTACGTTG, contig AAAAC, k = 3, min_count 1: AAA is new (left
    neighbour A once; right neighbours A and C: a fork), AAC is in both and
    keeps the reads' count 1."""
    bases, offs = flat([b"ACGTACGTTG"])
    c, co = flat([b"AAAAC"])
    res = oracle.merge_contigs(bases, b"I" * 10, offs, oracle.Params(k=3, min_count=1), c, co)
    assert [x.decode() for x in res.keys] == ["AAA", "AAC", "ACG", "CAA", "GTA"]
    assert list(res.count) == [0, 1, 4, 1, 2]
    assert tuple(res.cls[0]) == (0, oracle.FORK)
    assert list(res.ext[0]) == [0] * 8


def test_merge_with_no_contigs_changes_nothing():
    rs = synth.generate(synth.SINGLE_GENOME.scaled(300))
    p = oracle.Params(k=21)
    want = oracle.run(rs.bases, rs.quals, rs.offsets, p)
    got = oracle.merge_contigs(rs.bases, rs.quals, rs.offsets, p, b"", np.zeros(1, dtype=np.uint64))
    assert as_rows(got) == as_rows(want)


def test_merge_with_the_reads_as_contigs_adds_nothing_at_min_count_one():
    rs = synth.generate(synth.SINGLE_GENOME.scaled(200))
    p = oracle.Params(k=21, min_count=1)
    want = oracle.run(rs.bases, rs.quals, rs.offsets, p)
    got = oracle.merge_contigs(rs.bases, rs.quals, rs.offsets, p, rs.bases, rs.offsets)
    assert as_rows(got) == as_rows(want)


@pytest.mark.parametrize("seed", range(20))
def test_merge_against_brute_force(seed):
    rng = random.Random(3000 + seed)
    reads = random_reads(rng, rng.randint(0, 12), 1, 30, alphabet=rng.choice(["ACGT", "AC"]), n_rate=0.02)
    contigs = [r[0] for r in random_reads(rng, rng.randint(0, 6), 1, 40, alphabet=rng.choice(["ACGT", "AC"]),
                                          n_rate=0.02)]
    k = rng.choice([1, 3, 5, 7])
    p = oracle.Params(k=k, min_count=rng.choice([1, 2]), ext_mode=rng.choice([0, 1]))
    bases, offs = flat([r[0] for r in reads])
    quals = b"".join(r[1] for r in reads)
    c, co = flat(contigs)
    got = oracle.merge_contigs(bases, quals, offs, p, c, co)
    assert as_rows(got) == merge_brute(reads, contigs, p)


# ------------------------------------------------------ de Bruijn graph traversal
def rc_str(s):
    return "".join(COMP[c] for c in reversed(s))


def traverse_brute(keys, cls):
    """Sec. II-C written differently: each canonical k-mer with two UNIQUE
    sides has two ports (left, right); an oriented k-mer x links its right
    port to y = x[1..] + r(x) when y is another such k-mer naming x back
    (hairpins, x followed by its own reverse complement, link nothing).
    Components are chains or rings of ports; a chain is read from an end, a
    ring from its smallest k-mer in stored orientation."""
    keys = [x.decode() if isinstance(x, bytes) else x for x in keys]
    uu = {key: (int(c[0]), int(c[1])) for key, c in zip(keys, cls) if c[0] < 4 and c[1] < 4}

    def lr(x):
        c = min(x, rc_str(x))
        if c not in uu:
            return None
        l, r = uu[c]
        return (l, r) if c == x else (3 - r, 3 - l)

    def right(x):  # the oriented k-mer joined to x's right, or None
        s = lr(x)
        if s is None:
            return None
        y = x[1:] + ORDER[s[1]]
        t = lr(y)
        if t is None or ORDER[t[0]] != x[0] or min(y, rc_str(y)) == min(x, rc_str(x)):
            return None
        return y

    # port of oriented x's right side: (canonical, 1) if x is stored, else (canonical, 0)
    def rport(x):
        c = min(x, rc_str(x))
        return (c, 1 if c == x else 0)

    link = {}
    for c in uu:
        for x in (c, rc_str(c)):
            y = right(x)
            if y is not None:
                a, b = rport(x), rport(rc_str(y))  # y's left side is the right side of rc(y)
                link[a], link[b] = b, a
    out, seen = [], set()
    for c in sorted(uu):
        if c in seen:
            continue
        # walk out of the left port to the end of the chain (or once around a ring)
        v, p, ring = c, 0, False
        while (v, p) in link:
            v, q = link[(v, p)]
            p = 1 - q
            if v == c:
                ring = True
                break
        if ring:
            ring_members, v, p = [c], c, 1
            while True:
                v, q = link[(v, p)]
                p = 1 - q
                if v == c:
                    break
                ring_members.append(v)
            start, port = min(ring_members), 1
        else:
            start, port = v, 1 - p  # the end reached, leaving through its other port
        x = start if port == 1 else rc_str(start)
        s, v, p = x, start, port
        seen.add(start)
        while (v, p) in link:
            w, q = link[(v, p)]
            if w in seen:
                break
            seen.add(w)
            # w is read in stored orientation when entered through its left port
            y = w if q == 0 else rc_str(w)
            s += y[-1]
            v, p = w, 1 - q
        out.append(min(s, rc_str(s)))
    return sorted(out)


def genome_reads(g, L, step):
    return [(g[i:i + L], b"I" * L) for i in range(0, len(g) - L + 1, step)]


def test_traversal_of_one_genome_is_one_contig():
    """Error-free tiled reads of a sequence with no repeated 7-mer: every inner
    k-mer has unique extensions; the first and last k-mers have a dead end, so
    the contig is the genome without its first and last base."""
    g = b"ACGTTGCATGCCATAGGCTTACAGGATCCATTGACGGTACAT"
    res = oracle.run_reads(genome_reads(g, 20, 2), oracle.Params(k=7, min_count=1))
    want = g[1:-1]
    want = min(want, want.translate(bytes.maketrans(b"ACGT", b"TGCA"))[::-1])
    assert oracle.traverse(res.keys, res.cls) == [want]


def test_traversal_is_strand_symmetric():
    g = b"ACGTTGCATGCCATAGGCTTACAGGATCCATTGACGGTACAT"
    fwd = oracle.run_reads(genome_reads(g, 20, 2), oracle.Params(k=7, min_count=1))
    rcg = g.translate(bytes.maketrans(b"ACGT", b"TGCA"))[::-1]
    rev = oracle.run_reads(genome_reads(rcg, 20, 2), oracle.Params(k=7, min_count=1))
    assert oracle.traverse(fwd.keys, fwd.cls) == oracle.traverse(rev.keys, rev.cls)


def test_traversal_of_a_tandem_repeat_is_a_cycle():
    """Reads of a long period-7 repeat (no 5-mer equals another's reverse
    complement): seven k-mers in a ring; the contig is read from the smallest
    of them in stored orientation, one period plus k - 1 bases."""
    g = b"ACCGTTG" * 14
    res = oracle.run_reads(genome_reads(g, 40, 1), oracle.Params(k=5, min_count=1))
    got = oracle.traverse(res.keys, res.cls)
    assert len(res) == 7 and len(got) == 1 and len(got[0]) == 7 + 5 - 1
    assert got == [x.encode() for x in traverse_brute(res.keys, res.cls)]


def test_traversal_of_a_palindromic_repeat_uses_each_kmer_once():
    """A repeat whose reverse complement is a rotation of itself: a k-mer is
    followed by its own reverse complement (a hairpin), which joins nothing;
    every k-mer appears in exactly one contig."""
    g = b"ACGTTGCA" * 12
    res = oracle.run_reads(genome_reads(g, 40, 1), oracle.Params(k=5, min_count=1))
    got = oracle.traverse(res.keys, res.cls)
    assert got == [x.encode() for x in traverse_brute(res.keys, res.cls)]
    assert sum(len(c) - 5 + 1 for c in got) == len(res)


@pytest.mark.parametrize("seed", range(30))
def test_traversal_against_brute_force(seed):
    rng = random.Random(5000 + seed)
    k = rng.choice([3, 5, 7])
    # k-mer sets from a few random sequences read as tiled reads, plus random noise k-mers
    seqs = ["".join(rng.choice(ORDER) for _ in range(rng.randint(k + 2, 60))) for _ in range(rng.randint(1, 4))]
    reads = [(s.encode()[i:i + 15], b"I" * 15) for s in seqs for i in range(0, max(1, len(s) - 14), 3)]
    reads += random_reads(rng, rng.randint(0, 5), k, 20)
    res = oracle.run_reads(reads, oracle.Params(k=k, min_count=1, ext_mode=rng.choice([0, 1])))
    if len(res) == 0:
        return
    assert [c.decode() for c in oracle.traverse(res.keys, res.cls)] == traverse_brute(res.keys, res.cls)
