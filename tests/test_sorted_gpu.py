"""Sorted output (KMER_FLAG_SORTED_OUTPUT) against the oracle, row by row.

The oracle's records come out of an ordered map, in lexicographic order of
the k-mers, which is the numeric order of the 2-bit keys.  With the flag the
GPU's survivors must arrive in that same order, so no host-side sort is
applied here: row i of the GPU output equals row i of the oracle's.  The
radix sort works on 8-bit digits over the 2k key bits, so the k cover one,
two, three and four key words and odd digit counts (k = 21: 42 bits, 6
passes; k = 55: 110 bits, 14 passes; k = 127: 254 bits, 32 passes).
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1809_07014_gb300 as pkg
from tests.helpers import decode_keys

pytestmark = pytest.mark.gpu


def same_rows(got, want, label, distinct=True):
    gk = decode_keys(got.keys, got.k)
    assert len(gk) == len(want.keys), f"{label}: {len(gk)} survivors vs {len(want.keys)}"
    bad = np.nonzero(gk != want.keys)[0]
    assert bad.size == 0, f"{label}: order or keys differ from row {bad[:3]}: {gk[bad[:2]]} vs {want.keys[bad[:2]]}"
    assert (got.count == want.count).all(), f"{label}: counts differ"
    assert (got.ext == want.ext).all(), f"{label}: tallies differ"
    assert (got.cls == want.cls).all(), f"{label}: classes differ"
    assert got.windows == want.windows
    if distinct:
        assert got.distinct == want.distinct


def ascending(keys: np.ndarray) -> bool:
    """(n, W) words, word 0 most significant: strictly ascending rows."""
    if len(keys) < 2:
        return True
    a, b = keys[:-1], keys[1:]
    less = np.zeros(len(a), bool)
    eq = np.ones(len(a), bool)
    for w in range(keys.shape[1]):
        less |= eq & (a[:, w] < b[:, w])
        eq &= a[:, w] == b[:, w]
    return bool(less.all())


@pytest.fixture(scope="module")
def reads():
    import torch
    assert torch.cuda.is_available()
    return synth.generate(synth.METAGENOME_2G.scaled(40_000))


@pytest.mark.parametrize("k,min_count", [(21, 2), (31, 2), (33, 2), (55, 2), (63, 2), (99, 1), (127, 1)])
def test_sorted_rows_equal_the_oracle(reads, k, min_count):
    """(At k = 99 and 127 few k-mers of this low-coverage slice are seen twice;
    min_count 1 keeps every distinct k-mer, about 2 M.)"""
    r = pkg.ReadSet(reads.bases, reads.quals, reads.offsets)
    ka = pkg.KmerAnalysis(k, min_count=min_count, flags=pkg.KMER_FLAG_SORTED_OUTPUT | pkg.KMER_FLAG_PROFILE)
    ka.submit(r)
    got = ka.results()
    st = ka.stats()
    want = oracle.run_threads(reads.bases, reads.quals, reads.offsets, oracle.Params(k=k, min_count=min_count),
                              threads=oracle.host_threads())
    assert len(got) > 3 * 4096, "the case should span several sort tiles"
    assert ascending(got.keys)
    same_rows(got, want, f"sorted k={k}")
    assert st["n_sort"] == 1 and st["ms_sort"] > 0, st
    ka.close()
    r.close()


@pytest.mark.parametrize("variant,flags", [(pkg.KMER_VARIANT_HBM_TABLE, 0), (pkg.KMER_VARIANT_PARTITIONED,
                                                                             pkg.KMER_FLAG_BLOOM_GATE)])
def test_sorted_with_other_methods(reads, variant, flags):
    k = 31
    r = pkg.ReadSet(reads.bases, reads.quals, reads.offsets)
    ka = pkg.KmerAnalysis(k, variant=variant, flags=flags | pkg.KMER_FLAG_SORTED_OUTPUT)
    ka.submit(r)
    got = ka.results()
    want = oracle.run_threads(reads.bases, reads.quals, reads.offsets, oracle.Params(k=k),
                              threads=oracle.host_threads())
    same_rows(got, want, f"sorted, variant {variant}, flags {flags}", distinct=not flags)
    ka.close()
    r.close()


def test_sorted_into_caller_arrays(reads):
    """query_into device arrays (sorted in place there; misaligned arrays are
    refused before anything runs) and page-locked host arrays (staged through
    the analysis's buffers)."""
    import torch
    k = 33
    want = oracle.run_threads(reads.bases, reads.quals, reads.offsets, oracle.Params(k=k),
                              threads=oracle.host_threads())
    n, W = len(want.keys), 2
    r = pkg.ReadSet(reads.bases, reads.quals, reads.offsets)
    ka = pkg.KmerAnalysis(k, flags=pkg.KMER_FLAG_SORTED_OUTPUT)
    cap = n + 1000
    dk = torch.empty(cap * W, dtype=torch.int64, device="cuda")
    dc = torch.empty(cap, dtype=torch.int32, device="cuda")
    de = torch.empty(cap * 32 + 16, dtype=torch.uint8, device="cuda")
    dl = torch.empty(cap * 2 + 2, dtype=torch.uint8, device="cuda")
    ka.submit(r)
    for dext, dcls in ((4, 0), (0, 1)):  # host-side check: nothing is launched
        with pytest.raises(pkg.KmerError) as e:
            pkg.kmer_analysis_query_into(ka.handle, dk.data_ptr(), dc.data_ptr(), de.data_ptr() + dext,
                                         dl.data_ptr() + dcls, cap, pkg.KMER_DEVICE)
        assert e.value.code == pkg.KMER_ERR_INVALID_ARG
    v = pkg.kmer_analysis_query_into(ka.handle, dk.data_ptr(), dc.data_ptr(), de.data_ptr(), dl.data_ptr(),
                                     cap, pkg.KMER_DEVICE)
    assert v.n == n
    got = pkg.Result(k, dk[:n * W].cpu().numpy().view(np.uint64).reshape(n, W),
                     dc[:n].cpu().numpy().view(np.uint32),
                     de[:n * 32].cpu().numpy().view(np.uint32).reshape(n, 8),
                     dl[:2 * n].cpu().numpy().reshape(n, 2), int(v.windows), int(v.distinct))
    same_rows(got, want, "sorted into device arrays")
    # page-locked host arrays
    hk = torch.empty(cap * W, dtype=torch.int64).pin_memory()
    hc = torch.empty(cap, dtype=torch.int32).pin_memory()
    he = torch.empty(cap * 8, dtype=torch.int32).pin_memory()
    hl = torch.empty(cap * 2, dtype=torch.uint8).pin_memory()
    ka.reset()
    ka.submit(r)
    v = pkg.kmer_analysis_query_into(ka.handle, hk.data_ptr(), hc.data_ptr(), he.data_ptr(), hl.data_ptr(), cap,
                                     pkg.KMER_HOST)
    got = pkg.Result(k, hk[:n * W].numpy().view(np.uint64).reshape(n, W), hc[:n].numpy().view(np.uint32),
                     he[:n * 8].numpy().view(np.uint32).reshape(n, 8), hl[:2 * n].numpy().reshape(n, 2),
                     int(v.windows), int(v.distinct))
    same_rows(got, want, "sorted into page-locked host arrays")
    ka.close()
    r.close()


def test_sorted_merge_and_tiny_sets(reads):
    """Merge keeps the order (the contig-only k-mers are sorted in); empty,
    one-survivor and two-survivor results pass through the sort unchanged."""
    k = 31
    rng = np.random.default_rng(5)
    pieces = [reads.bases[int(reads.offsets[i]):int(reads.offsets[i + 1])].tobytes() for i in range(300)]
    pieces.append(rng.choice(np.frombuffer(b"ACGT", np.uint8), 4000).tobytes())
    contigs = np.frombuffer(b"".join(pieces), np.uint8).copy()
    offs = np.zeros(len(pieces) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(p) for p in pieces], dtype=np.uint64)
    r = pkg.ReadSet(reads.bases, reads.quals, reads.offsets)
    ka = pkg.KmerAnalysis(k, flags=pkg.KMER_FLAG_SORTED_OUTPUT)
    ka.submit(r)
    ka.query()
    got = ka.merge_contigs(contigs, offs)
    want = oracle.merge_contigs(reads.bases, reads.quals, reads.offsets, oracle.Params(k=k), contigs, offs)
    same_rows(got, want, "sorted merge")
    assert (got.count == 0).any()
    rec = ka.lookup(got.keys[::97])  # the index is rebuilt over the sorted positions
    assert rec["found"].all() and (rec["count"] == got.count[::97]).all()
    ka.close()
    r.close()
    # tiny sets: one read of 8, 9 and 10 bases at k = 9 and min_count 1
    seq = b"GATTACACC"
    for L, n_want in ((8, 0), (9, 1), (10, 2)):
        s = (seq + b"T")[:L]
        b = np.frombuffer(s, np.uint8).copy()
        quals = np.full(L, 33 + 40, np.uint8)
        o = np.array([0, L], np.uint64)
        ka = pkg.KmerAnalysis(9, min_count=1, flags=pkg.KMER_FLAG_SORTED_OUTPUT)
        ka.submit_raw(b, quals, o)
        got = ka.results()
        want = oracle.run(b, quals, o, oracle.Params(k=9, min_count=1))
        assert len(got) == n_want
        same_rows(got, want, f"tiny {s!r}")
        ka.close()
