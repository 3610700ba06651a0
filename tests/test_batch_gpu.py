"""Batched analyses (many samples, uneven sizes, mixed k) give, job by job,
exactly the regular create/submit/query result -- and the oracle's."""
import numpy as np
import pytest

import oracle
import synth
import paper_1809_07014_gb300 as pkg
from tests.helpers import assert_same

pytestmark = pytest.mark.gpu


def sample(i, n_reads):
    return synth.generate(synth.metagenome_sample(i, n_reads * 150, n_genomes=3 + i % 5).scaled(
        n_reads, genome_len_min=20_000 + 7000 * i, genome_len_max=40_000 + 9000 * i))


@pytest.fixture(scope="module")
def samples():
    import torch
    assert torch.cuda.is_available()
    sizes = [300, 5000, 1200, 20000, 800, 9000, 150, 3000]
    return [sample(i, n) for i, n in enumerate(sizes)]


def regular(rs_obj, k):
    ka = pkg.KmerAnalysis(k)
    ka.submit(rs_obj)
    r = ka.results()
    ka.close()
    return r


def same_result(a, b):
    ka, kb = a.keys, b.keys
    oa = np.lexsort(ka.T[::-1]) if len(ka) else np.arange(0)
    ob = np.lexsort(kb.T[::-1]) if len(kb) else np.arange(0)
    assert len(oa) == len(ob)
    assert np.array_equal(ka[oa], kb[ob]) and np.array_equal(a.count[oa], b.count[ob])
    assert np.array_equal(a.ext[oa], b.ext[ob]) and np.array_equal(a.cls[oa], b.cls[ob])
    assert a.windows == b.windows and a.distinct == b.distinct


def test_batch_matches_regular_and_oracle(samples):
    ks = [21, 33, 55, 21, 33, 55, 21, 33]
    rsets = [pkg.ReadSet(s.bases, s.quals, s.offsets) for s in samples]
    b = pkg.Batch([(r, {"k": k}) for r, k in zip(rsets, ks)])
    b.run()
    st = b.stats()
    assert st["jobs"] == len(samples) and st["graph_launches"] == st["waves"] >= 1
    for i, (r, k) in enumerate(zip(rsets, ks)):
        same_result(b.results(i), regular(r, k))
    for i in (0, 2, 4):  # a few jobs against the oracle as well
        s = samples[i]
        assert_same(b.results(i), oracle.run(s.bases, s.quals, s.offsets, oracle.Params(k=ks[i])), f"job {i}")
    # replaying the graphs gives the same results
    first = [b.results(i) for i in range(len(samples))]
    b.run()
    for i in range(len(samples)):
        same_result(b.results(i), first[i])
    b.close()


def test_batch_waves_and_output_repairs(samples):
    """A small memory budget splits the jobs into several waves; a tiny survivor
    hint makes outputs overflow, and those jobs are repaired inside their wave
    (output grown, leaves re-run) with exact results."""
    ks = [21, 21, 33, 55, 33, 21, 55, 33]
    rsets = [pkg.ReadSet(s.bases, s.quals, s.offsets) for s in samples]
    jobs = [(r, {"k": k, "survivors_hint": 1 if i % 3 == 0 else 0}) for i, (r, k) in enumerate(zip(rsets, ks))]
    b = None
    for mb in (96, 80, 72, 64, 56, 48, 40):  # the first budget that still holds the outputs but splits the jobs
        try:
            cand = pkg.Batch(jobs, memory_budget=mb << 20)
        except pkg.KmerError as e:
            assert e.code == pkg.KMER_ERR_OOM
            continue
        if cand.stats()["waves"] >= 2:
            b = cand
            break
        cand.close()
    assert b is not None, "no budget split the jobs into waves"
    b.run()
    st = b.stats()
    assert st["waves"] >= 2 and st["jobs_repaired"] >= 1 and st["jobs_alone"] == 0
    for i, (r, k) in enumerate(zip(rsets, ks)):
        same_result(b.results(i), regular(r, k))
    # the second run may re-plan from the first run's counts (and repair under
    # the new plan); after that the plan and the repaired descriptors hold
    b.run()
    for i, (r, k) in enumerate(zip(rsets, ks)):
        same_result(b.results(i), regular(r, k))
    replans = b.stats()["replans"]
    b.run()
    st = b.stats()
    assert st["jobs_repaired"] == 0 and st["jobs_alone"] == 0 and st["replans"] == replans
    for i, (r, k) in enumerate(zip(rsets, ks)):
        same_result(b.results(i), regular(r, k))
    b.close()


def test_batch_repairs_leaf_layout_in_wave(samples):
    """Heavy-hitter reads overflow level-2 leaves (but not the level-1 buckets):
    the job gets an exact leaf layout and its repartition re-runs inside the
    wave; the result equals the regular analysis and the oracle."""
    s = samples[3]
    heavy = np.frombuffer(bytes(s.bases[:150]), np.uint8)
    n_heavy = 3000
    bases = np.concatenate([s.bases, np.tile(heavy, n_heavy)])
    quals = np.concatenate([s.quals, np.tile(s.quals[:150], n_heavy)])
    offsets = np.concatenate([s.offsets, s.offsets[-1] + 150 * np.arange(1, n_heavy + 1, dtype=np.uint64)])
    r = pkg.ReadSet(bases, quals, offsets)
    b = pkg.Batch([(r, {"k": 21, "leaf_bits": 12, "l1_bits": 2})])
    b.run()
    st = b.stats()
    assert st["jobs_repaired"] == 1 and st["jobs_alone"] == 0, st
    assert_same(b.results(0), oracle.run(bases, quals, offsets, oracle.Params(k=21)), "heavy hitters")
    b.run()  # the exact layout is kept (and the job keeps its plan)
    assert b.stats()["jobs_repaired"] == 0 and b.stats()["replans"] == 0
    assert_same(b.results(0), oracle.run(bases, quals, offsets, oracle.Params(k=21)), "heavy hitters, rerun")
    b.close()


def test_batch_of_empty_and_tiny_jobs():
    reads = [(b"ACGTACGTACGTACGTACGTACGTA", b"I" * 25), (b"ACG", b"III")]
    bases = np.frombuffer(b"".join(x[0] for x in reads), np.uint8).copy()
    quals = np.frombuffer(b"".join(x[1] for x in reads), np.uint8).copy()
    offsets = np.array([0, 25, 28], np.uint64)
    r1 = pkg.ReadSet(bases, quals, offsets)
    r0 = pkg.ReadSet(np.zeros(0, np.uint8), np.zeros(0, np.uint8), np.zeros(1, np.uint64))
    b = pkg.Batch([(r0, {"k": 21}), (r1, {"k": 5, "min_count": 1}), (r1, {"k": 127})])
    b.run()
    assert len(b.results(0)) == 0 and len(b.results(2)) == 0
    assert_same(b.results(1), oracle.run(bases, quals, offsets, oracle.Params(k=5, min_count=1)), "tiny")
    b.close()


def test_batch_replans_from_its_counts(samples):
    """Hints far from the truth (100 distinct k-mers) give a coarse plan whose
    leaves overflow and are counted in key ranges; the run's counts re-plan
    the batch, and every run is exact."""
    ks = [21, 33, 55, 21]
    rsets = [pkg.ReadSet(s.bases, s.quals, s.offsets) for s in samples[:4]]
    b = pkg.Batch([(r, {"k": k, "distinct_hint": 100}) for r, k in zip(rsets, ks)])
    b.run()
    assert b.stats()["replans"] == 0
    first = [b.results(i) for i in range(4)]
    b.run()
    assert b.stats()["replans"] == 1
    for i, (r, k) in enumerate(zip(rsets, ks)):
        same_result(b.results(i), regular(r, k))
        same_result(first[i], regular(r, k))
    b.run()
    assert b.stats()["replans"] == 1  # the learned plan holds
    b.close()


def test_batch_job_of_100_mbases_complete_on_hash_shards():
    """One job of the batched workload at full size (107 Mbases, k = 33, 32
    genomes) in a batch with smaller jobs of mixed k: its survivors in the
    hash shards 0-3 of 16 (a quarter of the key space) equal the oracle's
    key by key, with every count, tally and class; the other jobs equal the
    regular path."""
    import bench
    from tests.helpers import fnv1a_keys, decode_keys
    recipes = bench.batch_workload(1.0)
    big_recipe, big_k = recipes[22]
    assert big_recipe.n_reads * 150 >= 100_000_000 and big_k == 33
    big = synth.generate(big_recipe, threads=oracle.host_threads())
    small = [(sample(i, n), k) for i, (n, k) in enumerate([(4000, 21), (700, 55), (12000, 33), (2500, 21)])]
    rsets = [pkg.ReadSet(big.bases, big.quals, big.offsets)] + [pkg.ReadSet(s.bases, s.quals, s.offsets)
                                                               for s, _ in small]
    ks = [big_k] + [k for _, k in small]
    b = pkg.Batch([(r, {"k": k}) for r, k in zip(rsets, ks)])
    b.run()
    got = b.results(0)
    for i in range(1, len(rsets)):
        same_result(b.results(i), regular(rsets[i], ks[i]))
    b.close()
    for r in rsets:
        r.close()
    lo, hi, n_shards = 0, 4, 16
    h = fnv1a_keys(decode_keys(got.keys, big_k)) % np.uint64(n_shards)
    sel = np.nonzero((h >= lo) & (h < hi))[0]
    want = oracle.run_threads(big.bases, big.quals, big.offsets, oracle.Params(k=big_k), lo, hi, n_shards,
                              threads=oracle.host_threads())
    assert len(want) > 500_000
    part = pkg.Result(keys=got.keys[sel], count=got.count[sel], ext=got.ext[sel], cls=got.cls[sel], k=big_k,
                      windows=want.windows, distinct=want.distinct)
    assert_same(part, want, f"107-Mbase batch job, k={big_k}, shards {lo}-{hi - 1} of {n_shards}")
