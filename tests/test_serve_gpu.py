"""Serving: requests that arrive while others run are admitted as memory
frees up and overlap on the device; every result is the same alone and in
the mix, and equal to the oracle's (exact: all integer)."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth
import paper_1809_07014_gb300 as pkg
from tests.helpers import assert_same
from tests.test_batch_gpu import same_result

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def readsets():
    import torch
    assert torch.cuda.is_available()
    out = []
    for i, n in enumerate([40000, 3000, 15000, 800, 25000, 6000]):
        s = synth.generate(synth.metagenome_sample(20 + i, n * 150, n_genomes=4 + i).scaled(
            n, genome_len_min=30_000, genome_len_max=90_000))
        r = pkg.ReadSet(s.bases, s.quals, s.offsets)
        r.src = s  # the reads themselves, for the oracle
        out.append(r)
    return out


def alone(rs, k):
    ka = pkg.KmerAnalysis(k)
    ka.submit(rs)
    r = ka.results()
    ka.close()
    return r


REQUESTS = [(0, 21), (1, 33), (2, 55), (3, 77), (4, 99), (5, 21), (0, 33), (2, 21), (4, 55), (1, 21), (0, 21)]


def test_results_same_alone_and_in_the_mix(readsets):
    want = {i: alone(readsets[r], k) for i, (r, k) in enumerate(REQUESTS)}
    srv = pkg.Server(workers=4)
    ids = {}

    def client(part):
        for i in part:  # staggered arrivals from several threads
            r, k = REQUESTS[i]
            ids[i] = srv.submit(readsets[r], k)
            time.sleep(0.002 * (i % 3))

    threads = [threading.Thread(target=client, args=(list(range(j, len(REQUESTS), 3)),)) for j in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    infos = {}
    for i, rid in ids.items():
        got = srv.results(rid)
        same_result(got, want[i])
        infos[i] = srv.wait(rid)[1]
        assert infos[i]["status"] == 0 and infos[i]["t_done_ms"] >= infos[i]["t_start_ms"] >= infos[i]["t_submit_ms"]
        srv.release(rid)
    st = srv.stats()
    assert st["completed"] == len(REQUESTS) and st["failed"] == 0
    assert st["peak_running"] >= 2, "requests never overlapped"
    srv.close()


ORACLE_REQUESTS = [(1, 33), (3, 77), (5, 99), (2, 55), (0, 21), (5, 21), (3, 99), (1, 77), (4, 33), (2, 21)]


def test_served_results_equal_the_oracle(readsets):
    """Staggered requests from three client threads, mixed k (one to four
    words per key), four workers: every served result equals the oracle on
    that request's reads, element by element."""
    srv = pkg.Server(workers=4)
    ids = {}

    def client(part):
        for i in part:
            r, k = ORACLE_REQUESTS[i]
            ids[i] = srv.submit(readsets[r], k)
            time.sleep(0.003 * (1 + i % 4))

    threads = [threading.Thread(target=client, args=(list(range(j, len(ORACLE_REQUESTS), 3)),)) for j in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    got = {}
    for i, rid in ids.items():
        got[i] = srv.results(rid)
        srv.release(rid)
    st = srv.stats()
    assert st["completed"] == len(ORACLE_REQUESTS) and st["failed"] == 0
    assert st["peak_running"] >= 2, "requests never overlapped"
    srv.close()
    for i, (r, k) in enumerate(ORACLE_REQUESTS):
        s = readsets[r].src
        want = oracle.run_threads(s.bases, s.quals, s.offsets, oracle.Params(k=k), threads=oracle.host_threads())
        assert_same(got[i], want, f"served request {i} (readset {r}, k={k})")


def test_admission_by_footprint_queues_and_stays_exact(readsets):
    """A budget that holds about one large request at a time: later requests wait
    for releases (pending) and reuse pooled analyses; results stay exact."""
    srv = pkg.Server(memory_budget=600 << 20, workers=3)
    reqs = [(0, 21), (4, 21), (0, 21), (2, 33), (4, 21)]
    ids = [srv.submit(readsets[r], k) for r, k in reqs]
    assert srv.stats()["pending"] >= 1
    for rid, (r, k) in zip(ids, reqs):
        same_result(srv.results(rid), alone(readsets[r], k))
        srv.release(rid)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    srv.close()


def test_bad_request_rejected(readsets):
    srv = pkg.Server(workers=1)
    with pytest.raises(pkg.KmerError) as e:
        srv.submit(readsets[0], 22)
    assert e.value.code == pkg.KMER_ERR_INVALID_ARG
    srv.close()


def test_pooled_analysis_serves_other_readsets_at_the_same_k(readsets):
    """A released analysis is reused by a later request with the same result
    parameters (same k) on another readset of another size; the server's
    learned distinct ratio sizes it, and the result is exact."""
    srv = pkg.Server(workers=1)
    rid = srv.submit(readsets[0], 21)
    srv.wait(rid)
    srv.release(rid)
    assert srv.stats()["pooled"] == 1
    for i in (3, 2):
        rid = srv.submit(readsets[i], 21)
        srv.wait(rid)
        assert srv.stats()["pooled"] == 0  # the pooled analysis was taken
        same_result(srv.results(rid), alone(readsets[i], 21))
        srv.release(rid)
    srv.close()


def test_threads_pipelining_staged_steps():
    """Host threads each with their own stream, readset and analysis, as the
    end-to-end bench runs them: reads re-packed from page-locked memory by the
    copy engines, counting one step at a time under a lock, survivors copied
    out by the copy engines.  Every step of every thread gives the oracle's
    result for its own reads."""
    import torch
    import oracle
    from tests.helpers import assert_same
    samples = [synth.generate(synth.METAGENOME_2G.scaled(6_000 + 1_000 * i, seed=40 + i)) for i in range(3)]
    want = [oracle.run(s.bases, s.quals, s.offsets, oracle.Params(k=31)) for s in samples]
    lock, errors = threading.Lock(), []

    def lane(i):
        try:
            st = torch.cuda.Stream()
            s = samples[i]
            b, q, o = (torch.from_numpy(a).pin_memory() for a in (s.bases, s.quals, s.offsets.view(np.int64)))
            rs = pkg.ReadSet(b[:150].clone(), q[:150].clone(), torch.tensor([0, 150], dtype=torch.int64), stream=st,
                             staged=True)
            ka = pkg.KmerAnalysis(31, stream=st)
            for step in range(3):
                rs.pack(b, q, o, stream=st, staged=True)
                with lock:
                    ka.reset()
                    ka.submit(rs)
                    v = pkg.kmer_analysis_query(ka.handle)
                n = int(v.n)
                keys, cnt = np.empty((n, 1), np.uint64), np.empty(n, np.uint32)
                ext, cls = np.empty((n, 8), np.uint32), np.empty((n, 2), np.uint8)
                pkg.kmer_analysis_copy_results(ka.handle, keys.ctypes.data, cnt.ctypes.data, ext.ctypes.data,
                                               cls.ctypes.data, n)
                got = pkg.Result(31, keys, cnt, ext, cls, int(v.windows), int(v.distinct))
                assert_same(got, want[i], f"thread {i} step {step}")
            ka.close()
            rs.close()
        except Exception as e:  # reported in the main thread
            errors.append(e)

    ths = [threading.Thread(target=lane, args=(i,)) for i in range(3)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    assert not errors, errors


def test_threads_with_different_fanouts(readsets):
    """Host threads that analyse at the same time with different partition
    fan-outs launch the same kernels with different shared-memory sizes; the
    kernels' shared-memory limit is one process-wide attribute, which no
    thread may lower under another (a full-size serving run once failed a
    scatter launch that way).  Every result equals the one taken alone."""
    import torch
    rs = readsets[0]
    want = alone(rs, 31)
    shapes = [(6, 0), (12, 3), (16, 11), (20, 9), (14, 7), (18, 11), (10, 0), (22, 11)]
    errors = []

    def worker(t):
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                for i in range(12):
                    leaf_bits, l1_bits = shapes[(t + i) % len(shapes)]
                    ka = pkg.KmerAnalysis(31, stream=stream, leaf_bits=leaf_bits, l1_bits=l1_bits)
                    ka.submit(rs)
                    got = ka.results()
                    ka.close()
                    try:
                        same_result(got, want)
                    except AssertionError:
                        errors.append(f"thread {t}, leaf_bits {leaf_bits}, l1_bits {l1_bits}: results differ")
        except Exception as e:  # collected: pytest sees only the main thread's failures
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors[:3]
