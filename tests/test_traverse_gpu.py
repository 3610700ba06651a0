"""De Bruijn graph traversal (Sec. II-C) on the GPU against the oracle: the
contigs formed by k-mers with unique extensions, over a query's survivors and
over a set merged with contig k-mers."""
import numpy as np
import pytest

import oracle
import synth
import paper_1809_07014_gb300 as pkg
from tests.helpers import decode_keys

pytestmark = pytest.mark.gpu


def gpu_contigs(ka):
    return sorted(ka.traverse())


def oracle_contigs(res, k):
    return oracle.traverse(decode_keys(res.keys, k), res.cls)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.mark.parametrize("k", [21, 31, 55, 77])
def test_traversal_of_single_genome_reads(torch_cuda, k):
    """30x reads of a 100 kbp genome with 0.5 % errors: long contigs broken at
    error forks."""
    rs = synth.generate(synth.SINGLE_GENOME)
    r = pkg.ReadSet(rs.bases, rs.quals, rs.offsets)
    ka = pkg.KmerAnalysis(k)
    ka.submit(r)
    res = ka.results()
    got = gpu_contigs(ka)
    want = oracle_contigs(res, k)
    assert len(want) > 10 and max(len(c) for c in want) > 1000
    assert got == want
    ka.close()
    r.close()


def test_traversal_of_a_metagenome_slice(torch_cuda):
    rs = synth.generate(synth.METAGENOME_2G.scaled(30_000))
    r = pkg.ReadSet(rs.bases, rs.quals, rs.offsets)
    ka = pkg.KmerAnalysis(31)
    ka.submit(r)
    res = ka.results()
    assert gpu_contigs(ka) == oracle_contigs(res, 31)
    ka.close()
    r.close()


def test_traversal_of_rings_and_hairpins(torch_cuda):
    """Error-free reads of tandem repeats: a period-7 ring (cut before its
    smallest k-mer) and a repeat whose reverse complement is a rotation of
    itself (hairpins), beside a plain sequence."""
    rng = np.random.default_rng(3)
    plain = rng.choice(np.frombuffer(b"ACGT", np.uint8), 600).tobytes()
    seqs = [b"ACCGTTG" * 30, b"ACGTTGCA" * 30, plain]
    reads = [s[i:i + 60] for s in seqs for i in range(0, len(s) - 59, 3)]
    bases = np.frombuffer(b"".join(reads), np.uint8).copy()
    quals = np.full(len(bases), ord("I"), np.uint8)
    offs = np.zeros(len(reads) + 1, np.uint64)
    offs[1:] = np.cumsum([len(x) for x in reads])
    for k in (5, 21):
        r = pkg.ReadSet(bases, quals, offs)
        ka = pkg.KmerAnalysis(k, min_count=1)
        ka.submit(r)
        res = ka.results()
        assert gpu_contigs(ka) == oracle_contigs(res, k)
        ka.close()
        r.close()


def test_traversal_after_merge(torch_cuda):
    """Contig k-mers merged into the set join the traversal (count 0, the
    classes of their contig neighbours)."""
    rs = synth.generate(synth.SINGLE_GENOME.scaled(4000))
    r = pkg.ReadSet(rs.bases, rs.quals, rs.offsets)
    ka = pkg.KmerAnalysis(21)
    ka.submit(r)
    ka.query()
    contigs = np.frombuffer(b"".join(rs.bases[int(rs.offsets[i]):int(rs.offsets[i + 1])].tobytes()
                                     for i in range(0, 400, 2)), np.uint8).copy()
    coffs = np.arange(0, 201, dtype=np.uint64) * 150
    merged = ka.merge_contigs(contigs, coffs)
    assert gpu_contigs(ka) == oracle_contigs(merged, 21)
    ka.close()
    r.close()
