"""Merge of Algorithm 1 (Sec. II-G) on the GPU against the oracle: the
survivors of a query merged with the k-mers of a contig set (ExtractKmers),
k-mers in both kept once with the reads' record, contig-only k-mers appended
with count 0 and the classes of their contig neighbours."""
import numpy as np
import pytest

import oracle
import synth
import paper_1809_07014_gb300 as pkg
from tests.helpers import assert_same, decode_keys

pytestmark = pytest.mark.gpu


def contig_set(reads, rng):
    """Contigs: 400 of the reads themselves (k-mers mostly shared with the
    survivors, their singletons new), long random contigs with N runs, a
    palindromic stretch and contigs shorter than k."""
    pieces = [reads.bases[int(reads.offsets[i]):int(reads.offsets[i + 1])].tobytes() for i in range(400)]
    for L in (3000, 5000, 1200):
        s = bytearray(rng.choice(np.frombuffer(b"ACGT", np.uint8), L).tobytes())
        s[L // 3:L // 3 + 5] = b"NNNNN"
        pieces.append(bytes(s))
    pieces += [b"ACGTACGTACGTACGTACGTACGTACGTACGT" * 8, b"ACG", b""]
    data = b"".join(pieces)
    offs = np.zeros(len(pieces) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(p) for p in pieces], dtype=np.uint64)
    return np.frombuffer(data, np.uint8).copy(), offs


@pytest.fixture(scope="module")
def reads():
    import torch
    assert torch.cuda.is_available()
    return synth.generate(synth.METAGENOME_2G.scaled(20_000))


@pytest.mark.parametrize("k", [21, 33, 55, 99])
def test_merge_matches_oracle(reads, k):
    rng = np.random.default_rng(k)
    contigs, offs = contig_set(reads, rng)
    r = pkg.ReadSet(reads.bases, reads.quals, reads.offsets)
    ka = pkg.KmerAnalysis(k)
    ka.submit(r)
    before = ka.results()
    got = ka.merge_contigs(contigs, offs)
    want = oracle.merge_contigs(reads.bases, reads.quals, reads.offsets, oracle.Params(k=k), contigs, offs)
    assert len(got) > len(before)
    assert_same(got, want, f"merge k={k}")
    # the appended k-mers come after the survivors, with count 0
    assert (got.count[len(before):] == 0).all() and (got.count[:len(before)] > 0).all()
    # lookups see the merged set
    new_keys = got.keys[len(before):len(before) + 50]
    rec = ka.lookup(new_keys)
    assert rec["found"].all() and (rec["count"] == 0).all()
    ka.close()
    r.close()


def test_merge_with_no_contigs_changes_nothing(reads):
    r = pkg.ReadSet(reads.bases, reads.quals, reads.offsets)
    ka = pkg.KmerAnalysis(31)
    ka.submit(r)
    before = ka.results()
    got = ka.merge_contigs(b"", np.zeros(1, dtype=np.uint64))
    assert len(got) == len(before)
    assert (decode_keys(got.keys, 31) == decode_keys(before.keys, 31)).all()
    ka.close()
    r.close()


def test_merge_from_device_contigs(reads):
    import torch
    rng = np.random.default_rng(7)
    contigs, offs = contig_set(reads, rng)
    r = pkg.ReadSet(reads.bases, reads.quals, reads.offsets)
    ka = pkg.KmerAnalysis(31)
    ka.submit(r)
    ka.query()
    got = ka.merge_contigs(torch.from_numpy(contigs).cuda(), torch.from_numpy(offs.view(np.int64)).cuda())
    want = oracle.merge_contigs(reads.bases, reads.quals, reads.offsets, oracle.Params(k=31), contigs, offs)
    assert_same(got, want, "merge from device contigs")
    ka.close()
    r.close()


@pytest.mark.parametrize("on_device", [False, True])
def test_merge_of_long_contigs(reads, on_device):
    """Contigs of 60 000 and 150 000 bases (and one made of 200 reads end to
    end): the library cuts them into overlapping pieces before extracting
    their k-mers, which must change no k-mer, class or count of the merge."""
    import torch
    rng = np.random.default_rng(11)
    pieces = [rng.choice(np.frombuffer(b"ACGT", np.uint8), L).tobytes() for L in (60_000, 150_000)]
    pieces.append(b"".join(reads.bases[int(reads.offsets[i]):int(reads.offsets[i + 1])].tobytes()
                           for i in range(200)))
    pieces.append(b"ACGT")
    contigs = np.frombuffer(b"".join(pieces), np.uint8).copy()
    offs = np.zeros(len(pieces) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(p) for p in pieces], dtype=np.uint64)
    for k in (31, 55):
        r = pkg.ReadSet(reads.bases, reads.quals, reads.offsets)
        ka = pkg.KmerAnalysis(k)
        ka.submit(r)
        ka.query()
        if on_device:
            got = ka.merge_contigs(torch.from_numpy(contigs).cuda(), torch.from_numpy(offs.view(np.int64)).cuda())
        else:
            got = ka.merge_contigs(contigs, offs)
        want = oracle.merge_contigs(reads.bases, reads.quals, reads.offsets, oracle.Params(k=k), contigs, offs)
        assert_same(got, want, f"long contigs, k={k}, device={on_device}")
        ka.close()
        r.close()
