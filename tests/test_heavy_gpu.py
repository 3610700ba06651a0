"""Heavy hitters (Sec. II-B: a few k-mers seen very often load one owner):
one read in 20 of a metagenome slice replaced by a homopolymer, so that one
k-mer fills a leaf far past the shared-memory table's 65 536 records and one
level-1 bucket far past the others.  Repeated queries on one handle stay
exact and keep their memory: the hot leaf is recounted in HBM with
warp-aggregated updates and laid out exactly, without widening every leaf."""
import numpy as np
import pytest

import oracle
import synth
import paper_1809_07014_gb300 as pkg
from tests.helpers import assert_same

pytestmark = pytest.mark.gpu


def test_heavy_hitter_repeated_queries():
    import torch
    assert torch.cuda.is_available()
    rs = synth.generate(synth.METAGENOME_2G.scaled(200_000))
    b = rs.bases.reshape(-1, 150)
    q = rs.quals.reshape(-1, 150)
    b[::20] = ord("A")
    q[::20] = ord("I")
    want = oracle.run_threads(rs.bases, rs.quals, rs.offsets, oracle.Params(k=31), threads=oracle.host_threads())
    r = pkg.ReadSet(rs.bases, rs.quals, rs.offsets)
    ka = pkg.KmerAnalysis(31)
    dev = []
    for i in range(4):
        ka.reset()
        ka.submit(r)
        got = ka.results()
        st = ka.stats()
        assert_same(got, want, f"heavy hitter, query {i}")
        assert st["fallback_leaves"] >= 1, st
        dev.append(st["device_bytes"])
    top = int(np.argmax(got.count))
    assert int(got.count[top]) == (len(rs.offsets) - 1 + 19) // 20 * (150 - 30)
    assert dev[3] <= 1.25 * dev[1], dev  # the leaf slack did not grow query after query
    ka.close()
    r.close()
