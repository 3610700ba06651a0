"""CUDA path vs the CPU oracle, element by element (exact: all integer).

Every case runs through the C ABI (ctypes binding) on cuda:0 and compares the
sorted survivors (keys, counts, eight extension tallies, two classes) and the
window / distinct totals with the oracle on the same seeded reads.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1809_07014_gb300 as pkg
from tests.helpers import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch


@pytest.fixture(scope="module")
def single_genome():
    return synth.generate(synth.SINGLE_GENOME)


def run_gpu(rs, k, device=False, torch=None, **params):
    if device:
        dev = (torch.from_numpy(rs.bases).cuda(), torch.from_numpy(rs.quals).cuda(),
               torch.from_numpy(rs.offsets.view(np.int64)).cuda())
        r = pkg.ReadSet(*dev, qual_offset=params.get("qual_offset", 33),
                        qual_threshold=params.get("qual_threshold", 20))
    else:
        r = pkg.ReadSet(rs.bases, rs.quals, rs.offsets, qual_offset=params.get("qual_offset", 33),
                        qual_threshold=params.get("qual_threshold", 20))
    ka = pkg.KmerAnalysis(k, **params)
    ka.submit(r)
    res = ka.results()
    st = ka.stats()
    ka.close()
    r.close()
    return res, st


def oracle_params(k, **params):
    keep = {f: params[f] for f in ("min_count", "qual_offset", "qual_threshold", "ext_mode", "t_base",
                                   "err_num", "err_den", "t_ext") if f in params}
    return oracle.Params(k=k, **keep)


def check(rs, k, label, torch=None, device=False, **params):
    got, st = run_gpu(rs, k, device=device, torch=torch, **params)
    want = oracle.run(rs.bases, rs.quals, rs.offsets, oracle_params(k, **params))
    assert_same(got, want, f"{label} k={k} {params}")
    return got, st


# ------------------------------------------------------------ workloads
def test_single_genome_k21(torch_cuda, single_genome):
    """The single-genome workload (100 kbp, 20 000 x 150 bp reads, k = 21)."""
    _, st = check(single_genome, 21, "single genome", torch=torch_cuda, device=True)
    assert st["survivors"] > 50_000 and st["retries"] == 0


@pytest.mark.parametrize("k", [21, 33, 55, 77, 99])
def test_multi_k_resident_readset(torch_cuda, single_genome, k):
    """Iterative multi-k on the single-genome reads: one resident readset, W = 1..4."""
    check(single_genome, k, "multi-k", torch=torch_cuda, device=True)


def test_resident_readset_reused_across_k(torch_cuda, single_genome):
    rs = single_genome
    r = pkg.ReadSet(rs.bases, rs.quals, rs.offsets)
    for k in (21, 33, 55, 77, 99):
        ka = pkg.KmerAnalysis(k)
        ka.submit(r)
        assert_same(ka.results(), oracle.run(rs.bases, rs.quals, rs.offsets, oracle.Params(k=k)), f"k={k}")
        ka.close()
    r.close()


def test_metagenome_slice_k31(torch_cuda):
    """A 60 000-read slice of the 2-Gbase metagenome recipe (log-normal abundance,
    1 % errors with low qualities, N bases), k = 31: two partition levels."""
    rs = synth.generate(synth.METAGENOME_2G.scaled(60_000))
    got, st = check(rs, 31, "metagenome slice", leaf_bits=14)
    assert st["l2_bits"] > 0


@pytest.mark.parametrize("pinned", [True, False])
def test_staged_host_reads(torch_cuda, pinned):
    """Reads moved to the device by the copy engines (KMER_HOST_STAGED) from
    page-locked or pageable host memory, packed into a reused readset: the
    oracle's results."""
    rs = synth.generate(synth.METAGENOME_2G.scaled(20_000, seed=21))
    b, q, o = (torch_cuda.from_numpy(a) for a in (rs.bases, rs.quals, rs.offsets.view(np.int64)))
    if pinned:
        b, q, o = b.pin_memory(), q.pin_memory(), o.pin_memory()
    r = pkg.ReadSet(b[:1000].clone(), q[:1000].clone(), torch_cuda.tensor([0, 1000], dtype=torch_cuda.int64),
                    staged=True)
    r.pack(b, q, o, staged=True)
    ka = pkg.KmerAnalysis(31)
    ka.submit(r)
    got = ka.results()
    ka.close()
    r.close()
    assert_same(got, oracle.run(rs.bases, rs.quals, rs.offsets, oracle.Params(k=31)), "staged reads")


@pytest.mark.parametrize("variant", [pkg.KMER_VARIANT_PARTITIONED, pkg.KMER_VARIANT_HBM_TABLE])
@pytest.mark.parametrize("k", [1, 3, 15, 31, 33, 61, 63, 65, 95, 97, 127])
def test_every_word_boundary(torch_cuda, k, variant):
    rs = synth.generate(synth.Recipe("ragged", seed=17, n_genomes=2, genome_len_min=3000, genome_len_max=5000,
                                     abundance_sigma=1.0, n_reads=1500, read_len_min=1, read_len_max=300,
                                     subst_rate=0.02, err_qual_lo=2, err_qual_hi=12, n_rate=0.003))
    check(rs, k, "ragged", variant=variant)


@pytest.mark.parametrize("mode,extra", [
    (0, dict(t_base=0, err_num=1, err_den=20)), (0, dict(t_base=5, err_num=3, err_den=10)),
    (1, dict(t_ext=1)), (1, dict(t_ext=3)),
])
def test_classification_modes(torch_cuda, single_genome, mode, extra):
    sub = synth.generate(synth.SINGLE_GENOME.scaled(5000))
    check(sub, 25, "modes", ext_mode=mode, **extra)


@pytest.mark.parametrize("min_count,qt", [(1, 20), (3, 20), (2, 0), (2, 35), (5, 30)])
def test_thresholds(torch_cuda, min_count, qt):
    sub = synth.generate(synth.SINGLE_GENOME.scaled(4000))
    check(sub, 21, "thresholds", min_count=min_count, qual_threshold=qt)


# ---------------------------------------------------------- edge cases
def test_empty_readset(torch_cuda):
    ka = pkg.KmerAnalysis(21)
    r = pkg.ReadSet(np.zeros(0, np.uint8), np.zeros(0, np.uint8), np.zeros(1, np.uint64))
    ka.submit(r)
    res = ka.results()
    assert len(res) == 0 and res.windows == 0
    # no submit at all
    ka2 = pkg.KmerAnalysis(21)
    assert len(ka2.results()) == 0
    ka.close(); ka2.close(); r.close()


def test_short_and_all_n_reads(torch_cuda):
    reads = [(b"ACGT", b"IIII"), (b"N" * 200, b"#" * 200), (b"", b""), (b"ACGTNACGTACGTACGTACGTAN", b"I" * 23)]
    bases = np.frombuffer(b"".join(r[0] for r in reads), np.uint8).copy()
    quals = np.frombuffer(b"".join(r[1] for r in reads), np.uint8).copy()
    offsets = np.concatenate([[0], np.cumsum([len(r[0]) for r in reads])]).astype(np.uint64)
    for k in (5, 21, 23):
        ka = pkg.KmerAnalysis(k, min_count=1)
        r = pkg.ReadSet(bases, quals, offsets)
        ka.submit(r)
        want = oracle.run(bases, quals, offsets, oracle.Params(k=k, min_count=1))
        assert_same(ka.results(), want, f"short k={k}")
        ka.close(); r.close()


def test_heavy_hitter_exact_counts(torch_cuda):
    """A homopolymer k-mer seen 100 000 times (16-bit tallies would wrap): the
    leaf is recounted exactly in HBM."""
    L, n = 150, 800
    reads = [(b"A" * L, b"I" * L)] * n
    bases = np.frombuffer(b"".join(r[0] for r in reads), np.uint8).copy()
    quals = np.frombuffer(b"".join(r[1] for r in reads), np.uint8).copy()
    offsets = (np.arange(n + 1, dtype=np.uint64) * L)
    ka = pkg.KmerAnalysis(21)
    r = pkg.ReadSet(bases, quals, offsets)
    ka.submit(r)
    res = ka.results()
    assert ka.stats()["fallback_leaves"] >= 1
    assert len(res) == 1 and int(res.count[0]) == n * (L - 20)
    assert list(res.ext[0]) == [n * (L - 21), 0, 0, 0, n * (L - 21), 0, 0, 0]
    ka.close(); r.close()


def test_deep_coverage_tallies(torch_cuda):
    """A 3 kbp genome at about 300x: counts and per-side tallies in the
    hundreds (a tally far above any that low-coverage tests reach)."""
    rs = synth.generate(synth.SINGLE_GENOME.scaled(6_000, genome_len_min=3_000, genome_len_max=3_000, seed=11))
    got, _ = check(rs, 31, "deep coverage", torch=torch_cuda)
    assert int(got.count.max()) > 200 and int(got.ext.max()) > 128


def test_homopolymer_in_shared_table_leaf(torch_cuda):
    """One k-mer seen 13 000 times among 20 000 others (its leaf has fewer
    than 65 536 records): its left-A and right-A tallies are exact."""
    L, n = 150, 100
    hp = [(b"A" * L, b"I" * L)] * n
    other = synth.generate(synth.SINGLE_GENOME.scaled(200, seed=12))
    bases = np.concatenate([np.frombuffer(b"".join(r[0] for r in hp), np.uint8), other.bases])
    quals = np.concatenate([np.frombuffer(b"".join(r[1] for r in hp), np.uint8), other.quals])
    offsets = np.concatenate([np.arange(n, dtype=np.uint64) * L, other.offsets.astype(np.uint64) + n * L])
    got, _ = check(_Reads(bases, quals, offsets), 21, "homopolymer", torch=torch_cuda)
    a = got.count.argmax()
    assert int(got.count[a]) == n * (L - 20)


class _Reads:
    def __init__(self, bases, quals, offsets):
        self.bases, self.quals, self.offsets = bases, quals, offsets


def test_fallback_when_leaves_do_not_fit(torch_cuda):
    """Too few partitions for the distinct k-mers: leaves overflow the shared
    table and are recounted in HBM; results stay exact."""
    rs = synth.generate(synth.METAGENOME_2G.scaled(20_000))
    _, st = check(rs, 31, "forced fallback", leaf_bits=4)
    assert st["fallback_leaves"] > 0


def test_leaves_split_into_key_ranges(torch_cuda):
    """Leaves with more distinct k-mers than a shared table holds (but fewer
    than 65 536 records) are counted in key ranges, split by the next bits of
    the mixed key, instead of going to the HBM recount; results stay exact."""
    rs = synth.generate(synth.METAGENOME_2G.scaled(20_000))
    _, st = check(rs, 31, "key ranges", leaf_bits=7)
    assert st["leaf_splits"] > 0 and st["fallback_leaves"] == 0, st
    _, st = check(rs, 55, "key ranges, two words", leaf_bits=7)
    assert st["leaf_splits"] > 0, st


def test_many_passes(torch_cuda):
    rs = synth.generate(synth.METAGENOME_2G.scaled(20_000))
    _, st = check(rs, 31, "passes", memory_budget=8 << 20)
    assert st["passes"] > 1


def test_repeated_submits_commute(torch_cuda):
    """Submitting the reads in three chunks (in any order) gives the same result
    as one submit (update-only inserts commute)."""
    rs = synth.generate(synth.METAGENOME_2G.scaled(9000))
    want = oracle.run(rs.bases, rs.quals, rs.offsets, oracle.Params(k=31))
    cuts = [0, 2000, 6500, rs.n_reads]
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        o = rs.offsets[a:b + 1] - rs.offsets[a]
        s, e = int(rs.offsets[a]), int(rs.offsets[b])
        parts.append(pkg.ReadSet(rs.bases[s:e].copy(), rs.quals[s:e].copy(), o.copy()))
    ka = pkg.KmerAnalysis(31)
    for p in (parts[2], parts[0], parts[1]):
        ka.submit(p)
    assert_same(ka.results(), want, "chunked submits")
    # submit_raw path and a second query after reset
    ka.reset()
    ka.submit_raw(rs.bases, rs.quals, rs.offsets)
    assert_same(ka.results(), want, "submit_raw")
    ka.close()
    for p in parts:
        p.close()


def test_qual_mismatch_rejected(torch_cuda):
    rs = synth.generate(synth.SINGLE_GENOME.scaled(100))
    r = pkg.ReadSet(rs.bases, rs.quals, rs.offsets, qual_threshold=30)
    ka = pkg.KmerAnalysis(21)
    with pytest.raises(pkg.KmerError) as e:
        ka.submit(r)
    assert e.value.code == pkg.KMER_ERR_INVALID_ARG
    ka.close(); r.close()


def test_decreasing_offsets_rejected(torch_cuda):
    bases = np.frombuffer(b"ACGTACGTAC", np.uint8).copy()
    quals = np.full(10, 73, np.uint8)
    with pytest.raises(pkg.KmerError) as e:
        pkg.ReadSet(bases, quals, np.array([0, 6, 4, 10], np.uint64))
    assert e.value.code == pkg.KMER_ERR_INVALID_ARG
    import torch
    with pytest.raises(pkg.KmerError) as e:
        pkg.ReadSet(torch.from_numpy(bases).cuda(), torch.from_numpy(quals).cuda(),
                    torch.tensor([0, 6, 4, 10], dtype=torch.int64).cuda())
    assert e.value.code == pkg.KMER_ERR_INVALID_ARG
