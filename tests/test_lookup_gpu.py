"""Point lookups among the survivors (kmer_analysis_lookup): every survivor
is found in either orientation with its own count, tallies and classes;
k-mers that are not survivors are not found; the oracle's counts agree."""
import numpy as np
import pytest

import oracle
import synth
import paper_1809_07014_gb300 as pkg

pytestmark = pytest.mark.gpu

COMP = bytes.maketrans(b"ACGT", b"TGCA")


def encode(strings, k):
    """k-mer strings -> (n, W) uint64 words, word 0 most significant."""
    W = (2 * k + 63) // 64
    code = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}
    out = np.zeros((len(strings), W), dtype=np.uint64)
    for i, s in enumerate(strings):
        v = 0
        for ch in s:
            v = (v << 2) | code[ch]
        for w in range(W):
            out[i, W - 1 - w] = np.uint64((v >> (64 * w)) & 0xFFFFFFFFFFFFFFFF)
    return out


def decode(keys, k):
    W = keys.shape[1]
    res = []
    for row in keys:
        v = 0
        for w in range(W):
            v = (v << 64) | int(row[w])
        res.append(bytes(b"ACGT"[(v >> (2 * (k - 1 - i))) & 3] for i in range(k)))
    return res


@pytest.fixture(scope="module")
def sample():
    return synth.generate(synth.metagenome_sample(7, 3000 * 150, n_genomes=4).scaled(
        3000, genome_len_min=20_000, genome_len_max=40_000))


@pytest.mark.parametrize("k", [21, 33, 77, 99])
def test_lookup_survivors_both_orientations(sample, k):
    ka = pkg.KmerAnalysis(k)
    rs = pkg.ReadSet(sample.bases, sample.quals, sample.offsets)
    ka.submit(rs)
    res = ka.results()
    assert len(res) > 0
    rec = ka.lookup(res.keys)
    assert rec["found"].all() and not rec["flipped"].any()
    assert np.array_equal(rec["count"], res.count)
    assert np.array_equal(rec["ext"], res.ext) and np.array_equal(rec["cls"], res.cls)
    # reverse complements: same vertex, flipped
    strings = decode(res.keys[:500], k)
    rc = encode([s.translate(COMP)[::-1] for s in strings], k)
    rec = ka.lookup(rc)
    assert rec["found"].all() and rec["flipped"].all()
    assert np.array_equal(rec["count"], res.count[:500])
    # k-mers that are not survivors: random keys, and the singletons the oracle reports with min_count 1
    orc1 = oracle.run(sample.bases, sample.quals, sample.offsets, oracle.Params(k=k, min_count=1))
    singles = [s for s, c in zip(orc1.keys, orc1.count) if c == 1][:500]
    rec = ka.lookup(encode(singles, k))
    assert not rec["found"].any() and (rec["count"] == 0).all()
    rng = np.random.default_rng(k)
    rnd = ["".join(rng.choice(list("ACGT"), k)).encode() for _ in range(300)]
    have = set(decode(res.keys, k))
    canon = [min(s, s.translate(COMP)[::-1]) for s in rnd]
    rec = ka.lookup(encode(rnd, k))
    assert np.array_equal(rec["found"].astype(bool), np.array([c in have for c in canon]))
    # the oracle's counts for survivors it reports
    orc = oracle.run(sample.bases, sample.quals, sample.offsets, oracle.Params(k=k))
    pick = list(orc.keys[:200])
    rec = ka.lookup(encode(pick, k))
    assert rec["found"].all() and np.array_equal(rec["count"].astype(np.uint64), orc.count[:200])
    ka.close()
    rs.close()


def test_lookup_rejects_before_a_query_and_reuses_its_index(sample):
    ka = pkg.KmerAnalysis(31)
    with pytest.raises(pkg.KmerError) as e:
        ka.lookup(np.zeros((1, 1), np.uint64))
    assert e.value.code == pkg.KMER_ERR_BAD_STATE
    rs = pkg.ReadSet(sample.bases, sample.quals, sample.offsets)
    ka.submit(rs)
    res = ka.results()
    a = ka.lookup(res.keys[:10])
    b = ka.lookup(res.keys[:10])
    assert np.array_equal(a, b) and a["found"].all()
    # a key with bits above 2k is not a k-mer: not found
    bad = res.keys[:1].copy()
    bad[0, 0] |= np.uint64(1) << np.uint64(63)
    assert not ka.lookup(bad)["found"].any()
    ka.close()
    rs.close()


def test_query_into_caller_buffers(sample):
    """Survivors written straight into caller arrays: page-locked host memory
    or device memory give the regular query's results, and so do pageable
    host arrays filled by the copy engines (KMER_HOST_STAGED); a too small
    capacity, or pageable host memory to be written in place, is refused."""
    import torch
    rs = pkg.ReadSet(sample.bases, sample.quals, sample.offsets)
    for k in (31, 55):
        ka = pkg.KmerAnalysis(k)
        ka.submit(rs)
        ref = ka.results()
        n, W = len(ref), (2 * k + 63) // 64
        for where, dev in ((pkg.KMER_HOST, None), (pkg.KMER_DEVICE, "cuda"), (pkg.KMER_HOST_STAGED, "pageable"),
                           (pkg.KMER_HOST_STAGED, None)):
            if dev is None:
                mk = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
            elif dev == "pageable":
                mk = lambda shape, dt: torch.empty(shape, dtype=dt)
            else:
                mk = lambda shape, dt: torch.empty(shape, dtype=dt, device="cuda")
            cap = n + 17
            keys, cnt = mk((cap, W), torch.int64), mk(cap, torch.int32)
            ext, cls = mk((cap, 8), torch.int32), mk((cap, 2), torch.uint8)
            ka.reset()
            ka.submit(rs)
            v = pkg.kmer_analysis_query_into(ka.handle, keys.data_ptr(), cnt.data_ptr(), ext.data_ptr(),
                                             cls.data_ptr(), cap, where)
            assert int(v.n) == n and int(v.windows) == ref.windows and int(v.distinct) == ref.distinct
            got = pkg.Result(k, keys[:n].cpu().numpy().view(np.uint64), cnt[:n].cpu().numpy().view(np.uint32),
                             ext[:n].cpu().numpy().view(np.uint32), cls[:n].cpu().numpy(), ref.windows, ref.distinct)
            from tests.test_batch_gpu import same_result
            same_result(got, ref)
            # lookups and copies read the caller's arrays
            rec = ka.lookup(ref.keys[:50])
            assert rec["found"].all() and np.array_equal(rec["count"], ref.count[:50])
        # too small a capacity, and pageable host memory, are refused
        small = [torch.empty((max(1, n // 2), W), dtype=torch.int64).pin_memory(),
                 torch.empty(max(1, n // 2), dtype=torch.int32).pin_memory(),
                 torch.empty((max(1, n // 2), 8), dtype=torch.int32).pin_memory(),
                 torch.empty((max(1, n // 2), 2), dtype=torch.uint8).pin_memory()]
        for where in (pkg.KMER_HOST, pkg.KMER_HOST_STAGED):
            ka.reset()
            ka.submit(rs)
            with pytest.raises(pkg.KmerError) as e:
                pkg.kmer_analysis_query_into(ka.handle, *[t.data_ptr() for t in small], max(1, n // 2), where)
            assert e.value.code == pkg.KMER_ERR_INVALID_ARG
        pageable = [np.empty((n, W), np.uint64), np.empty(n, np.uint32), np.empty((n, 8), np.uint32),
                    np.empty((n, 2), np.uint8)]
        ka.reset()
        ka.submit(rs)
        with pytest.raises(pkg.KmerError) as e:
            pkg.kmer_analysis_query_into(ka.handle, *[a.ctypes.data for a in pageable], n, pkg.KMER_HOST)
        assert e.value.code == pkg.KMER_ERR_INVALID_ARG
        ka.close()
    rs.close()
