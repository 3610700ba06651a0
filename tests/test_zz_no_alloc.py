"""The allocation-free entry point (for callers that cannot call cudaMalloc,
e.g. code inside an allocator hook or a plugin whose host owns all device
memory) gives the same k-mers, counts, tallies and classes as the regular
create/submit/query entry point.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  Calls in a row use different inputs and
key widths (one, two, three and four words) so that each call shows the
shared static scratch is cleared between calls.
"""
import numpy as np
import pytest

import synth
import paper_1809_07014_gb300 as pkg

pytestmark = pytest.mark.gpu


def noalloc(torch, rs, k, offsets=None):
    bases = torch.from_numpy(rs.bases).cuda()
    quals = torch.from_numpy(rs.quals).cuda()
    offs = rs.offsets if offsets is None else offsets
    offsets = torch.from_numpy(np.ascontiguousarray(offs).view(np.int64)).cuda()
    cap = max(16, rs.n_bases)
    W = (2 * k + 63) // 64
    keys = torch.empty((cap, W), dtype=torch.int64, device="cuda")
    count = torch.empty(cap, dtype=torch.int32, device="cuda")
    ext = torch.empty((cap, 8), dtype=torch.int32, device="cuda")
    cls = torch.empty((cap, 2), dtype=torch.uint8, device="cuda")
    params = pkg.make_params(k)
    stream = torch.cuda.current_stream().cuda_stream
    n = pkg.kmer_analysis_run_noalloc(bases.data_ptr(), quals.data_ptr(), offsets.data_ptr(), rs.n_reads, params,
                                      keys.data_ptr(), count.data_ptr(), ext.data_ptr(), cls.data_ptr(), cap,
                                      stream)
    torch.cuda.synchronize()
    return (keys[:n].cpu().numpy().view(np.uint64), count[:n].cpu().numpy().view(np.uint32),
            ext[:n].cpu().numpy().view(np.uint32), cls[:n].cpu().numpy())


def regular(rs, k):
    r = pkg.ReadSet(rs.bases, rs.quals, rs.offsets)
    ka = pkg.KmerAnalysis(k)
    ka.submit(r)
    res = ka.results()
    ka.close()
    r.close()
    return res.keys, res.count, res.ext, res.cls


def by_key(keys, *cols):
    order = np.lexsort(keys.T[::-1])
    return (keys[order],) + tuple(c[order] for c in cols)


def test_noalloc_matches_regular_entry_point_two_calls_in_a_row():
    import torch
    assert torch.cuda.is_available()
    first = synth.generate(synth.SINGLE_GENOME.scaled(2000))
    second = synth.generate(synth.Recipe("mix", seed=9, n_genomes=3, genome_len_min=2000, genome_len_max=4000,
                                         abundance_sigma=1.0, n_reads=2400, subst_rate=0.01, err_qual_lo=2,
                                         err_qual_hi=12, n_rate=0.001))
    # three- and four-word keys (k >= 65) take at most 196 608 bases: 1300 reads of 150
    third = synth.generate(synth.Recipe("mix-wide", seed=10, n_genomes=2, genome_len_min=3000,
                                        genome_len_max=5000, abundance_sigma=1.0, n_reads=1300, subst_rate=0.01,
                                        err_qual_lo=2, err_qual_hi=12, n_rate=0.001))
    assert third.n_bases <= 196_608
    for rs, k in ((first, 21), (second, 33), (third, 77), (third, 99)):
        got = by_key(*noalloc(torch, rs, k))
        want = by_key(*regular(rs, k))
        assert len(got[0]) == len(want[0]) > 0
        for g, w in zip(got, want):
            assert np.array_equal(g, w)


def test_noalloc_rejects_inputs_beyond_its_static_table():
    import torch
    rs = synth.generate(synth.SINGLE_GENOME.scaled(3000))  # 450 000 bases > 393 216
    with pytest.raises(pkg.KmerError) as e:
        noalloc(torch, rs, 21)
    assert e.value.code == pkg.KMER_ERR_INVALID_ARG


def test_noalloc_rejects_decreasing_offsets():
    """A decreasing interior offset is refused before any base of that read is
    read: the input spans no more than the static table allows, and only one
    read's offsets are out of order."""
    import torch
    rs = synth.generate(synth.SINGLE_GENOME.scaled(2000))  # 300 000 bases, within the limit for k <= 63
    offs = rs.offsets.copy()
    offs[1000] = offs[999] - 1  # read 999 would end before it starts, read 1000 starts before read 999
    with pytest.raises(pkg.KmerError) as e:
        noalloc(torch, rs, 21, offsets=offs)
    assert e.value.code == pkg.KMER_ERR_INVALID_ARG
    # the entry point still works on good input afterwards
    got = by_key(*noalloc(torch, rs, 21))
    want = by_key(*regular(rs, 21))
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
