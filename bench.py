#!/usr/bin/env python
"""Throughput of k-mer analysis on one GB300: canonical k-mers per second.

Workload: the synthetic metagenome of 50 genomes (1-5 Mbp, log-normal
abundance sigma 1.5), 13 333 334 reads x 150 bp = 2 Gbases, 1 % substitutions
with low qualities, 0.01 % N; k = 31, count threshold 2, quality threshold 20.
A step is the whole hot path on one batch: pack the reads (a1), roll
canonical k-mers and partition them (a2-a3), count, filter, classify and
compact (a4-a7).  `value` counts valid k-mer windows per second with the
reads resident in HBM; `e2e` is the same through the C ABI from pinned host
buffers, host->device copy of the reads and device->host copy of every
surviving k-mer included.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank analyses its own sample (its own seed):
independent problems, no collective on the data path, weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "canonical k-mers/sec"
UNIT = "k-mers/s"
ORACLE_SAMPLE_READS = 200_000  # cpu_baseline sample: about 10-20 s of oracle work on every host core
REF_STEP_READS = 60_000        # reference arm: reads per timed step (a few seconds each on every host core)
EXTRA_SCALE = 0.25             # sub-records of the default line: batched and served workloads at this size
EXTRA_REQUESTS = 24


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--k", type=int, default=31)
    ap.add_argument("--reads", type=int, default=0, help="override the number of reads (development only)")
    ap.add_argument("--variant", choices=["partitioned", "hbm_table"], default="partitioned")
    ap.add_argument("--leaf-bits", type=int, default=0)
    ap.add_argument("--gate", action="store_true", help="single: Bloom gate (k-mers seen once kept out of counting)")
    ap.add_argument("--sorted", action="store_true", help="single: survivors in ascending key order")
    ap.add_argument("--mode", choices=["single", "batched", "serve", "multik", "large", "assembly"], default="single",
                    help="single: the 2-Gbase metagenome (default line); batched: 64 samples of uneven size and "
                         "mixed k in one graph per wave; serve: Poisson arrivals through the serving loop")
    ap.add_argument("--scale", type=float, default=1.0, help="batched/serve: scale every sample size")
    ap.add_argument("--tune", choices=["auto", "hints", "none"], default="auto",
                    help="batched: autotuned geometry and hints, sizing hints only, or no hints")
    ap.add_argument("--requests", type=int, default=40, help="serve: number of requests")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-threads", type=int, default=3, help="host threads of the end-to-end pipeline")
    ap.add_argument("--e2e-steps", type=int, default=24,
                    help="end-to-end steps of the several-thread run (at least --steps): the pipeline "
                         "fills and drains once per run")
    ap.add_argument("--e2e-repeats", type=int, default=3, help="end-to-end runs of the several-thread pipeline "
                                                                "(the median is reported)")
    ap.add_argument("--e2e-io", choices=["staged", "in-place"], default="staged",
                    help="end to end with several threads: host buffers moved by the copy engines "
                         "(KMER_HOST_STAGED, the counting of one step at a time) or read and written in "
                         "place by the kernels (KMER_HOST)")
    ap.add_argument("--e2e-alloc", choices=["torch", "huge"], default="huge",
                    help="end to end: page-locked host buffers from torch's allocator, or anonymous memory "
                         "advised for 512 MB transparent huge pages and registered with the driver")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="single: leave out the batched, serving and multi-k sub-records of the default line")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def load_peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Source files of each kernel's device code: its .cu and the device headers it
# includes (kernels.h holds only host-side declarations and helpers).
KERNEL_SOURCES = {
    "pack_kernel": ["pack.cu", "common.cuh"],
    "scatter_kernel": ["scatter.cu", "stage.cuh", "roll.cuh", "common.cuh"],
    "repart_kernel": ["repart.cu", "stage.cuh", "common.cuh"],
    "leaf_kernel": ["leaf.cu", "roll.cuh", "common.cuh"],
    "direct_insert_kernel": ["hbm.cu", "roll.cuh", "common.cuh"],
    "gate_kernel": ["gate.cu", "roll.cuh", "common.cuh"],
}


def kernel_source_sha(name: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[name]:
        h.update(open(os.path.join(ROOT, "paper_1809_07014_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kernel_traffic(name: str, src: str = ""):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, or None
    when the summary is missing or the kernel's sources changed since."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    if not os.path.exists(path) or name not in KERNEL_SOURCES:
        return None
    text = open(path).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_bytes = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.e+]+)", text)
    if not m_sha or not m_bytes:
        return None
    return float(m_bytes.group(1)) if kernel_source_sha(name) == m_sha.group(1) else None


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=self.tmp,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.tmp.flush()
        rows = [r.split(",") for r in open(self.tmp.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def hash_form_bytes_per_window(k: int, read_len: int, windows: int, distinct: int, survivors: int) -> float:
    """Algorithmic DRAM bytes per window of k-mer analysis in its hash-table
    form, the fixed denominator for every variant: the packed input, one
    table sector read and write-back per window, the table sweep and the
    survivors' output."""
    W = (2 * k + 63) // 64
    inp = 0.5 * read_len / max(1, read_len - k + 1)
    table = 64.0 if W == 1 else 96.0
    sweep = distinct * (8 * W + 4 + 16) / max(1, windows)
    out = survivors * (8 * W + 4 + 32 + 2) / max(1, windows)
    return inp + table + sweep + out


def rank_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def reduce_over_ranks(seconds: float, windows: int, device) -> tuple[float, int]:
    """Whole-job figures: the slowest rank's timed region and the windows all
    ranks analysed (each rank runs its own sample; nothing else is exchanged)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return seconds, windows
    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([windows], device=device, dtype=torch.int64)
    dist.all_reduce(w)
    return float(t.item()), int(w.item())


def workload(rank: int, n_reads: int):
    import synth
    r = synth.METAGENOME_2G
    if rank:
        r = synth.Recipe(f"{r.name}-rank{rank}", seed=r.seed + 1000 * rank, n_genomes=r.n_genomes,
                         genome_len_min=r.genome_len_min, genome_len_max=r.genome_len_max,
                         abundance_sigma=r.abundance_sigma, n_reads=r.n_reads, subst_rate=r.subst_rate,
                         err_qual_lo=r.err_qual_lo, err_qual_hi=r.err_qual_hi, n_rate=r.n_rate)
    if n_reads:
        r = r.scaled(n_reads)
    return r


def oracle_rate(rs, k: int, n_reads: int):
    """The oracle (as it stands) on the first n_reads reads, in its sharded mode
    on every host core: shard s of S keeps the keys whose FNV-1a hash is s mod
    S, one shard per core, each shard walking every read.  Returns windows/s,
    seconds, windows, reads and cores."""
    import oracle
    n_reads = min(n_reads, rs.n_reads)
    end = int(rs.offsets[n_reads])
    cores = oracle.host_threads()
    t0 = time.perf_counter()
    parts = oracle.run_shards(rs.bases[:end], rs.quals[:end], rs.offsets[:n_reads + 1], oracle.Params(k=k),
                              range(cores), cores, cores)
    dt = time.perf_counter() - t0
    windows = sum(p.windows for p in parts)
    return windows / dt, dt, windows, n_reads, cores


def config_of(args, recipe, n_bases):
    return {"workload": f"synthetic metagenome, {recipe.n_genomes} genomes, {n_bases / 1e9:.2f} Gbases, "
                        f"150 bp reads, k={args.k}",
            "reads": recipe.n_reads, "bases": n_bases, "read_len": 150, "k": args.k, "min_count": 2,
            "qual_threshold": 20, "variant": args.variant, "bloom_gate": bool(args.gate),
            "sorted_output": bool(args.sorted),
            "l2": "inputs (reads 4 GB, records >12 GB) larger than the 129 MB L2; no flush"}


# ------------------------------------------------- page-locked host buffers
_HUGE = 512 << 20  # the largest transparent huge page here (64 KB base pages)
_KEEP = []         # mappings registered with the driver, kept for the process
_HUGE_FAILED = []  # registrations the driver refused


def pinned(shape, dtype, huge: bool):
    """A page-locked host array.  huge: anonymous memory aligned to 512 MB and
    advised for transparent huge pages, then registered with the driver, so
    that the copy engines translate few large pages; else torch's pinned
    allocator."""
    import mmap
    import ctypes
    import numpy as np
    import torch
    n = int(np.prod(shape)) * np.dtype(dtype).itemsize
    if not huge or n < _HUGE:
        return torch.empty(shape, dtype=getattr(torch, np.dtype(dtype).name)).pin_memory()
    size = (n + _HUGE - 1) // _HUGE * _HUGE
    m = mmap.mmap(-1, size + _HUGE, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    base = ctypes.addressof(ctypes.c_char.from_buffer(m))
    lead = (-base) % _HUGE
    if hasattr(mmap, "MADV_HUGEPAGE"):
        m.madvise(mmap.MADV_HUGEPAGE, lead, size)
    arr = np.frombuffer(m, dtype=np.uint8, count=size, offset=lead)
    arr[::65536] = 0  # fault the pages in
    rc = torch.cuda.cudart().cudaHostRegister(base + lead, size, 0)
    if int(rc) != 0:  # not registered: torch's pinned allocator instead, and say so
        _HUGE_FAILED.append(str(rc))
        del arr
        try:
            m.close()
        except BufferError:
            pass
        return torch.empty(shape, dtype=getattr(torch, np.dtype(dtype).name)).pin_memory()
    _KEEP.append(m)
    return torch.from_numpy(arr[:n].view(dtype).reshape(shape))


# ------------------------------------------------------------- reference arm
def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return  # the oracle runs on rank 0 only
    import synth
    recipe = workload(0, args.reads)
    sample = workload(0, REF_STEP_READS)  # the first reads of the same recipe
    rs = synth.generate(sample)
    rates, wins, cores = [], 0, 1
    for i in range(args.warmup + args.steps):
        rate, dt, w, n, cores = oracle_rate(rs, args.k, REF_STEP_READS)
        if i >= args.warmup:
            rates.append(rate)
            wins += w
    value = statistics.median(rates)
    desc = (f"first {REF_STEP_READS} reads ({wins // max(1, args.steps)} windows) of the workload, "
            f"sharded oracle, one shard per host core ({cores})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * (wins / args.steps) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": config_of(args, recipe, 150 * recipe.n_reads),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_1809_07014_gb300 as pkg

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    recipe = workload(rank, args.reads)
    rs = synth.generate(recipe)
    n_bases = rs.n_bases
    bases_d = torch.from_numpy(rs.bases).to(dev)
    quals_d = torch.from_numpy(rs.quals).to(dev)
    offs_d = torch.from_numpy(rs.offsets.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream()
    variant = pkg.KMER_VARIANT_HBM_TABLE if args.variant == "hbm_table" else pkg.KMER_VARIANT_PARTITIONED

    rset = pkg.ReadSet(bases_d, quals_d, offs_d, stream=stream)
    gate_flag = pkg.KMER_FLAG_BLOOM_GATE if args.gate else 0
    if args.sorted:
        gate_flag |= pkg.KMER_FLAG_SORTED_OUTPUT
    ka = pkg.KmerAnalysis(args.k, stream=stream, flags=pkg.KMER_FLAG_PROFILE | gate_flag, variant=variant,
                          leaf_bits=args.leaf_bits)

    def step():
        rset.pack(bases_d, quals_d, offs_d, stream=stream)
        ka.reset()
        ka.submit(rset)
        return ka.query()

    # the first step is a cold query: a fresh handle allocates its buffers and,
    # with no earlier query at this k, plans its leaves from the window count
    first_ms = []
    for _ in range(max(args.warmup, 3 if args.warmup else 0)):
        torch.cuda.synchronize()
        tw = time.perf_counter()
        v = step()
        torch.cuda.synchronize()
        first_ms.append(1e3 * (time.perf_counter() - tw))
    stage_keys = ("ms_gate", "ms_scatter", "ms_repart", "ms_leaf", "ms_fallback", "ms_sort", "n_gate", "n_scatter",
                  "n_repart", "n_leaf", "n_fallback", "n_sort")
    acc = {k: 0.0 for k in stage_keys}
    launches = 0
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    windows = 0
    for _ in range(args.steps):
        v = step()
        st = ka.stats()
        for kk in stage_keys:
            acc[kk] += st[kk]
        launches += rset.launches + st["launches"]
        windows += int(v.windows)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    sec_max, tot_windows = reduce_over_ranks(e0.elapsed_time(e1) / 1e3, windows, dev)
    ms_max = 1e3 * sec_max
    value = tot_windows / sec_max
    st = ka.stats()
    n_surv = int(v.n)
    W = int(v.words)

    # ---- roofline of the dominant kernel (algorithmic bytes per launch / event time)
    n_reads = rs.n_reads
    n_blocks = int(((np.diff(rs.offsets) + np.uint64(31)) // np.uint64(32)).sum())
    rec = int(st["records_emitted"])
    out_bytes = n_surv * (8 * W + 4 + 32 + 2)
    alg = {
        "scatter_kernel": (n_blocks * 16 + 2 * 8 * (n_reads + 1) + rec * 8 * W, "scatter.cu", "n_scatter", "ms_scatter"),
        "repart_kernel": (2 * int(st["records_l2"]) * 8 * W, "repart.cu", "n_repart", "ms_repart"),
        "leaf_kernel": (rec * 8 * W + out_bytes, "leaf.cu", "n_leaf", "ms_leaf"),
    }
    if args.variant == "hbm_table":
        alg = {"direct_insert_kernel": (n_blocks * 16 + 2 * 8 * (n_reads + 1) + rec * 2 * 64, "hbm.cu",
                                        "n_scatter", "ms_scatter")}
    per_launch = {}
    for name, (bytes_, src, nkey, mskey) in alg.items():
        n = acc[nkey]
        if n:
            per_launch[name] = (bytes_, acc[mskey] / n, src)
    dom = max(per_launch, key=lambda kname: per_launch[kname][1])
    b, ms_l, src = per_launch[dom]
    peak, peak_kind = load_peaks()
    achieved = b / (ms_l / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": f"{peak_kind} copy bandwidth",
                "algorithmic_bytes_per_launch": b, "ms_per_launch": round(ms_l, 4),
                "traffic": kernel_traffic(dom, src),
                "stages_ms_per_step": {k[3:]: round(acc[k] / args.steps, 4) for k in stage_keys if k.startswith("ms_")}}
    # whole-path HBM fraction against the hash form's bytes per window
    bpw = hash_form_bytes_per_window(args.k, 150, int(st["windows"]), int(st["distinct"]), n_surv)
    per_gpu = value / world
    roofline["path_hbm_fraction"] = {"bytes_per_window": round(bpw, 2), "achieved": round(per_gpu * bpw / 1e9, 1),
                                     "frac": round(per_gpu * bpw / 1e9 / peak, 4),
                                     "note": "windows/s per GPU x hash-form bytes per window / peak (peak_kind)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config_of(args, recipe, n_bases), "roofline": roofline,
            "warmup_ms": {"cold_first_query": round(first_ms[0], 2) if first_ms else None,
                          "later": [round(x, 2) for x in first_ms[1:]],
                          "note": "host-timed warm-up steps; the first allocates and plans without history"}}

    # ---- end to end through the C ABI from pinned host buffers: every step packs
    # its reads from pinned host memory and copies its survivors into pinned
    # host memory.  Several host threads, each with its own readset, analysis
    # and stream, take turns.  Staged (the default): the reads and results
    # cross the host link by the copy engines (kmer_readset_pack with
    # KMER_HOST_STAGED, kmer_analysis_copy_results), and the counting itself
    # (kmer_analysis_query) runs one step at a time under a host lock, so one
    # step's kernels have the SMs while other steps' transfers run.  In place:
    # the kernels read and write the pinned buffers (KMER_HOST).  The
    # single-thread figure (in place) is reported beside.
    if not args.no_e2e:
        import threading
        ka.close()  # its device buffers go back to the pool for the two lanes below
        huge = args.e2e_alloc == "huge"
        b_h = pinned(rs.bases.shape, np.uint8, huge)
        b_h.copy_(torch.from_numpy(rs.bases))
        q_h = pinned(rs.quals.shape, np.uint8, huge)
        q_h.copy_(torch.from_numpy(rs.quals))
        o_h = torch.from_numpy(rs.offsets.view(np.int64)).pin_memory()
        cap = n_surv + n_surv // 8 + 1024
        n_thr = max(1, args.e2e_threads)
        staged = args.e2e_io == "staged"
        lanes = []
        for li in range(n_thr):
            st_l = torch.cuda.Stream(device=dev)
            lanes.append({
                "stream": st_l,
                "keys": pinned((cap, W), np.int64, huge),
                "cnt": pinned((cap,), np.int32, huge),
                "ext": pinned((cap, 8), np.int32, huge),
                "cls": pinned((cap, 2), np.uint8, huge),
                "rs": pkg.ReadSet(b_h, q_h, o_h, stream=st_l),
                "ka": pkg.KmerAnalysis(args.k, stream=st_l, variant=variant, leaf_bits=args.leaf_bits),
                "windows": 0, "d2h": 0})

        count_lock = threading.Lock()

        def e2e_step(ln, stg):
            # reads from pinned host buffers; survivors into pinned host buffers
            ln["rs"].pack(b_h, q_h, o_h, stream=ln["stream"], staged=stg)
            if stg:
                with count_lock:
                    ln["ka"].reset()
                    ln["ka"].submit(ln["rs"])
                    vv = pkg.kmer_analysis_query(ln["ka"].handle)
                pkg.kmer_analysis_copy_results(ln["ka"].handle, ln["keys"].data_ptr(), ln["cnt"].data_ptr(),
                                               ln["ext"].data_ptr(), ln["cls"].data_ptr(), cap)
            else:
                ln["ka"].reset()
                ln["ka"].submit(ln["rs"])
                vv = pkg.kmer_analysis_query_into(ln["ka"].handle, ln["keys"].data_ptr(), ln["cnt"].data_ptr(),
                                                  ln["ext"].data_ptr(), ln["cls"].data_ptr(), cap, pkg.KMER_HOST)
            ln["windows"] += int(vv.windows)
            ln["d2h"] += int(vv.n) * (8 * W + 4 + 32 + 2)

        cores = sorted(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else []

        def run_lane(ln, n, stg, idx=None):
            # each pipelining thread keeps a core of its own (it spins on its copies' events);
            # the ranks of one node take disjoint cores
            local_world = int(os.environ.get("LOCAL_WORLD_SIZE", "1"))
            if idx is not None and len(cores) >= local_world * (n_thr + 1):
                os.sched_setaffinity(0, {cores[local * (n_thr + 1) + 1 + idx]})
            torch.cuda.set_device(dev)
            for _ in range(n):
                e2e_step(ln, stg)

        for ln in lanes:  # warm-up: allocations and learned sizing
            e2e_step(ln, staged)
            e2e_step(ln, staged)
        e2e_step(lanes[0], False)
        torch.cuda.synchronize()
        # one thread, one step at a time, buffers read and written in place
        lanes[0]["windows"] = lanes[0]["d2h"] = 0
        barrier()
        t0 = time.perf_counter()
        run_lane(lanes[0], args.steps, False)
        torch.cuda.synchronize()
        dt1, w1 = reduce_over_ranks(time.perf_counter() - t0, lanes[0]["windows"], dev)
        # several threads taking turns; the run is repeated and its median reported
        # (the host side makes single runs vary)
        e2e_steps = max(args.steps, args.e2e_steps)
        reps = []
        for _ in range(max(1, args.e2e_repeats)):
            for ln in lanes:
                ln["windows"] = ln["d2h"] = 0
            barrier()
            t0 = time.perf_counter()
            ths = [threading.Thread(target=run_lane,
                                    args=(lanes[i], (e2e_steps + n_thr - 1 - i) // n_thr, staged, i))
                   for i in range(n_thr)]
            for th in ths:
                th.start()
            for th in ths:
                th.join()
            torch.cuda.synchronize()
            wins = sum(ln["windows"] for ln in lanes)
            dt_r, w_r = reduce_over_ranks(time.perf_counter() - t0, wins, dev)
            reps.append((w_r / dt_r, dt_r, w_r, sum(ln["d2h"] for ln in lanes)))
        rate2, dt2, w2, d2h = sorted(reps)[len(reps) // 2]
        h2d = 2 * n_bases + 8 * (n_reads + 1)
        line["e2e"] = {"value": rate2, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h // e2e_steps, "repeats": [round(r[0] / 1e9, 2) for r in reps],
                       "repeat_unit": "G k-mers/s", "median_of": len(reps),
                       "ms_per_step": 1e3 * dt2 / e2e_steps, "steps": e2e_steps, "host_threads": n_thr,
                       "host_io": ("KMER_HOST_STAGED (copy engines), one step counting at a time" if staged
                                   else "KMER_HOST (in place)"),
                       "host_buffers": ("anonymous memory advised for 512 MB transparent huge pages, registered "
                                        "with the driver" if args.e2e_alloc == "huge" and not _HUGE_FAILED
                                        else "torch pinned allocator" + (f" (registration refused: {_HUGE_FAILED[0]})"
                                                                         if _HUGE_FAILED else "")),
                       "one_thread": {"value": w1 / dt1, "ms_per_step": 1e3 * dt1 / args.steps,
                                      "host_io": "KMER_HOST (in place)"}}
        for ln in lanes:
            ln["ka"].close()
            ln["rs"].close()
    line["clocks"] = clocks.stop()
    line["gpu_launches"] = launches
    line["stats"] = {k: st[k] for k in ("windows", "distinct", "survivors", "passes", "l1_bits", "l2_bits",
                                        "retries", "fallback_leaves", "leaf_splits", "leaf_table_slots", "device_bytes")}

    # ---- CPU baseline: the oracle on a bounded sample, rank 0 at N = 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, dt, w, n, cores = oracle_rate(rs, args.k, ORACLE_SAMPLE_READS)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {n} reads ({w} windows) of the same workload, sharded oracle "
                                          f"(one FNV-1a shard per core, each walking every read), {dt:.1f} s on "
                                          f"{cores} host cores"}
    ka.close()
    if rank == 0 and world == 1 and not args.no_extras:
        line["assembly"] = assembly_record(rset, args.k, stream)
    rset.close()
    del bases_d, quals_d, offs_d
    # ---- the batched, served and multi-k forms on the same GPU (rank 0 at N = 1),
    # at reduced sizes so that the default run stays within minutes
    if rank == 0 and world == 1 and not args.no_extras:
        torch.cuda.synchronize()
        b = batched_record(EXTRA_SCALE, 3, 2, "hints")
        line["batched"] = {"value": b["value"], "unit": UNIT, "ms_per_run": round(b["ms_per_step"], 2),
                           "workload": b["config"]["workload"], "bases": b["config"]["bases"],
                           "single_instance": {"value": b["single_instance"]["value"],
                                               "ms_total": round(b["single_instance"]["ms_total"], 2)},
                           "speedup_vs_single_instance": round(b["speedup_vs_single_instance"], 4),
                           "waves": b["batch_stats"]["waves"], "graph_launches": b["batch_stats"]["graph_launches"],
                           "tuning": b["tuning"]}
        sv = serve_record(EXTRA_SCALE, EXTRA_REQUESTS)
        line["serve"] = {"value": sv["value"], "unit": UNIT, "latency_ms": sv["latency_ms"],
                         "workload": sv["config"]["workload"], "one_at_a_time": sv["one_at_a_time"]["value"],
                         "saturated": sv["saturated"]["value"], "peak_running": sv["peak_running"]}
        mk = multik_record(5, 3)
        line["multik"] = {"value": mk["value"], "unit": UNIT, "ms_per_round_batch": mk["batch"]["ms_per_round"],
                          "ms_per_round_sequential": mk["sequential"]["ms_per_round"],
                          "per_k_ms_sequential": mk["sequential"]["per_k_ms"], "workload": mk["config"]["workload"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# -------------------------------------------------------- assembly steps
def assembly_record(rset, k: int, stream, s_step: int = 2, reps: int = 3) -> dict:
    """The steps of Algorithm 1 around k-mer analysis, on the survivors of the
    bench workload (resident readset): the survivors sorted by key
    (KMER_FLAG_SORTED_OUTPUT, device time of the sort), the de Bruijn graph
    traversal into contigs (Sec. II-C), and the merge of those contigs'
    (k + s)-mers into the analysis at k + s (Sec. II-G).  Host-timed
    synchronous calls, median of `reps` after one warm-up."""
    import torch

    import paper_1809_07014_gb300 as pkg

    out = {}
    ka = pkg.KmerAnalysis(k, stream=stream, flags=pkg.KMER_FLAG_SORTED_OUTPUT | pkg.KMER_FLAG_PROFILE)
    ms_sort = []
    for i in range(reps + 1):
        ka.reset(); ka.submit(rset)
        v = ka.query()
        if i:
            ms_sort.append(ka.stats()["ms_sort"])
    n = int(v.n)
    out["sort"] = {"survivors": n, "ms": round(statistics.median(ms_sort), 3),
                   "keys_per_s": n / (statistics.median(ms_sort) / 1e3)}
    ms_trav = []
    for i in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cv = pkg.kmer_analysis_traverse(ka.handle)
        if i:
            ms_trav.append(1e3 * (time.perf_counter() - t0))
    out["traverse"] = {"k": k, "vertices_in": n, "contigs": int(cv.n_contigs), "contig_bases": int(cv.bases),
                       "ms": round(statistics.median(ms_trav), 3),
                       "k-mers_per_s": n / (statistics.median(ms_trav) / 1e3)}
    # merge the contigs' (k + s)-mers into the analysis at k + s
    k2 = k + s_step
    kb = pkg.KmerAnalysis(k2, stream=stream)
    ms_merge, added = [], 0
    for i in range(reps + 1):
        kb.reset(); kb.submit(rset)
        kb.query()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        added, mv = pkg.kmer_analysis_merge_contigs(kb.handle, cv.seq, cv.offsets, int(cv.n_contigs),
                                                   pkg.KMER_DEVICE)
        if i:
            ms_merge.append(1e3 * (time.perf_counter() - t0))
    contig_kmers = max(0, int(cv.bases) - int(cv.n_contigs) * (k2 - 1))
    out["merge"] = {"k": k2, "contigs": int(cv.n_contigs), "contig_windows_at_most": contig_kmers,
                    "added": int(added), "merged_set": int(mv.n), "ms": round(statistics.median(ms_merge), 3)}
    out["note"] = "host-timed synchronous calls (traverse, merge) and device time of the sort stage; median of 3"
    kb.close()
    ka.close()
    return out


def run_assembly(args):
    """The assembly sub-record alone: sort, traversal and merge on the bench
    workload's survivors (reads resident on the device)."""
    import numpy as np
    import torch

    import synth
    import paper_1809_07014_gb300 as pkg

    torch.cuda.set_device(0)
    recipe = workload(0, args.reads)
    rs = synth.generate(recipe)
    dev = [torch.from_numpy(a).cuda() for a in (rs.bases, rs.quals, rs.offsets.view(np.int64))]
    stream = torch.cuda.current_stream()
    rset = pkg.ReadSet(*dev, stream=stream)
    out = assembly_record(rset, args.k, stream)
    rset.close()
    print(json.dumps({"mode": "assembly", "config": config_of(args, recipe, rs.n_bases), **out}), flush=True)


# --------------------------------------------------------------- batched
BATCH_JOBS = 64


def batch_workload(scale: float):
    """64 samples: sizes log-uniform in [5 Mbases, 500 Mbases], k uniform in {21, 33, 55}."""
    import numpy as np
    import synth
    rng = np.random.default_rng(4)
    sizes = np.exp(rng.uniform(np.log(5e6), np.log(5e8), BATCH_JOBS)) * scale
    ks = rng.choice([21, 33, 55], BATCH_JOBS)
    recipes = []
    for i, (sz, k) in enumerate(zip(sizes, ks)):
        r = synth.metagenome_sample(i, int(sz), n_genomes=10 + i % 41)
        recipes.append((r.scaled(max(1, int(sz) // 150), genome_len_min=500_000, genome_len_max=2_000_000), int(k)))
    return recipes


def batched_record(scale: float, steps: int, warmup: int, tune: str) -> dict:
    """The 64-sample batch (one graph per wave) against the same jobs run as
    one regular query each, back to back, on the same GPU."""
    import numpy as np
    import torch

    import synth
    import paper_1809_07014_gb300 as pkg
    from paper_1809_07014_gb300.tune import autotune

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    recipes = batch_workload(scale)
    rsets, ks = [], []
    t0 = time.perf_counter()
    for r, k in recipes:
        s = synth.generate(r)
        rsets.append(pkg.ReadSet(s.bases, s.quals, s.offsets, stream=stream))
        ks.append(k)
    gen_s = time.perf_counter() - t0
    # one regular query per job: the single-instance baseline on the same GPU
    windows_all, t_single = 0, 0.0
    for rs, k in zip(rsets, ks):
        ka = pkg.KmerAnalysis(k, stream=stream)
        ka.submit(rs)
        ka.query()              # warm-up (allocations, learned sizing)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        v = ka.query()
        torch.cuda.synchronize()
        t_single += time.perf_counter() - t1
        windows_all += int(v.windows)
        ka.close()
    # autotune per k on the median-size job of that k
    tunings = {}
    if tune != "none":
        for k in sorted(set(ks)):
            idx = [i for i in range(len(ks)) if ks[i] == k]
            mid = sorted(idx, key=lambda i: rsets[i].n_bases)[len(idx) // 2]
            tunings[k] = autotune(rsets[mid], k, reps=1, stream=stream)
    jobs = []
    for rs, k in zip(rsets, ks):
        w = rs.n_bases  # windows of 150-bp reads are ~ (150-k+1)/150 of the bases
        w = int(w * (150 - k + 1) / 150)
        if tune == "none":
            jobs.append((rs, {"k": k}))
        elif tune == "hints":
            t = tunings[k].params(w)
            jobs.append((rs, {"k": k, "distinct_hint": t["distinct_hint"], "survivors_hint": t["survivors_hint"]}))
        else:
            jobs.append((rs, tunings[k].params(w)))
    b = pkg.Batch(jobs, stream=stream)
    for _ in range(max(2, warmup)):  # the first run may teach the batch its sizing (a re-plan)
        b.run()
    t1 = time.perf_counter()
    for _ in range(steps):
        b.run()
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t1) / steps
    st = b.stats()
    line = {"metric": METRIC, "value": windows_all / t_batch, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": 1e3 * t_batch, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"batched: {len(jobs)} synthetic metagenome samples, sizes log-uniform "
                                   f"{5 * scale:g}-{500 * scale:g} Mbases, k in {{21,33,55}}",
                       "bases": int(sum(r.n_bases for r in rsets)), "windows": windows_all, "tune": tune},
            "batch_stats": st,
            "single_instance": {"value": windows_all / t_single, "ms_total": 1e3 * t_single,
                                "note": "the same jobs, one regular query each, back to back"},
            "speedup_vs_single_instance": t_single / t_batch,
            "tuning": {k: {"keys_per_leaf": round(t.keys_per_leaf, 1), "l1_shift": t.l1_shift,
                           "distinct_ratio": round(t.distinct_ratio, 4), "method": t.method,
                           "method_ms": t.method_ms, "ms_best": round(t.ms_best, 3),
                           "ms_default": round(t.ms_default, 3)} for k, t in tunings.items()},
            "setup_s": round(gen_s, 1)}
    b.close()
    for rs in rsets:
        rs.close()
    return line


def run_batched(args):
    print(json.dumps(batched_record(args.scale, args.steps, args.warmup, args.tune)), flush=True)



# ----------------------------------------------------------------- serving
def pctl(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=float), q)) if xs else None


def serve_record(scale: float, n_requests: int) -> dict:
    """Serving: Poisson arrivals at 75 % of the measured one-at-a-time capacity,
    admitted by footprint on four workers; p50/p99 latency from submit to results."""
    import threading

    import numpy as np
    import torch

    import synth
    import paper_1809_07014_gb300 as pkg

    torch.cuda.set_device(0)
    rng = np.random.default_rng(5)
    n_pool = 12
    sizes = np.exp(rng.uniform(np.log(1e6), np.log(2e9), n_pool)) * scale
    pool = []
    t0 = time.perf_counter()
    for i, sz in enumerate(sizes):
        r = synth.metagenome_sample(5000 + i, int(sz), n_genomes=20)
        s = synth.generate(r.scaled(max(1, int(sz) // 150), genome_len_min=500_000, genome_len_max=2_000_000))
        pool.append(pkg.ReadSet(s.bases, s.quals, s.offsets))
    gen_s = time.perf_counter() - t0
    kset = [21, 33, 55, 77, 99]
    reqs = [(int(rng.integers(n_pool)), int(rng.choice(kset))) for _ in range(n_requests)]
    windows_of = lambda i, k: int(pool[i].n_bases * (150 - k + 1) / 150)
    # capacity: one request at a time, every request of the plan (warm analyses)
    srv = pkg.Server(workers=1)
    for i, k in reqs[:2]:  # warm-up: module loading and first allocations
        rid = srv.submit(pool[i], k)
        srv.wait(rid)
        srv.release(rid)
    t1 = time.perf_counter()
    alone_w = 0
    for i, k in reqs:
        rid = srv.submit(pool[i], k)
        v, _ = srv.wait(rid)
        alone_w += int(v.windows)
        srv.release(rid)
    t_alone = time.perf_counter() - t1
    srv.close()
    capacity = alone_w / t_alone                    # windows/s, one request at a time
    # saturated: every request queued at once, 4 workers overlapping on the device
    srv = pkg.Server(workers=4)
    t1 = time.perf_counter()
    sat_ids = [srv.submit(pool[i], k) for i, k in reqs]
    sat_w = 0
    for rid in sat_ids:
        v, _ = srv.wait(rid)
        sat_w += int(v.windows)
        srv.release(rid)
    t_sat = time.perf_counter() - t1
    peak_sat = srv.stats()["peak_running"]
    srv.close()
    mean_w = alone_w / len(reqs)
    rate = 0.75 * capacity / mean_w                 # requests/s
    gaps = rng.exponential(1.0 / rate, len(reqs))
    srv = pkg.Server(workers=4)
    ids = [None] * len(reqs)

    def client():
        start = time.perf_counter()
        at = 0.0
        for j, (i, k) in enumerate(reqs):
            at += gaps[j]
            d = start + at - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ids[j] = srv.submit(pool[i], k)

    th = threading.Thread(target=client)
    tstart = time.perf_counter()
    th.start()
    th.join()
    lat, first, last, tot_w = [], None, None, 0
    for j, rid in enumerate(ids):
        v, info = srv.wait(rid)
        lat.append(info["t_done_ms"] - info["t_submit_ms"])
        first = info["t_submit_ms"] if first is None else min(first, info["t_submit_ms"])
        last = info["t_done_ms"] if last is None else max(last, info["t_done_ms"])
        tot_w += int(v.windows)
        srv.release(rid)
    st = srv.stats()
    srv.close()
    span = (last - first) / 1e3
    line = {"metric": METRIC, "value": tot_w / span, "unit": UNIT, "n_gpus": 1, "steps": len(reqs), "warmup": 0,
            "ms_per_step": 1e3 * span / len(reqs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"serving: {len(reqs)} Poisson requests at 75% of measured capacity, sizes "
                                   f"log-uniform {scale:g}-{2000 * scale:g} Mbases, k in {kset}",
                       "pool_bases": int(sum(r.n_bases for r in pool)), "workers": 4},
            "latency_ms": {"p50": pctl(lat, 50), "p99": pctl(lat, 99), "max": max(lat)},
            "one_at_a_time": {"value": capacity, "note": "the same requests, one worker, back to back"},
            "saturated": {"value": sat_w / t_sat, "peak_running": peak_sat,
                          "note": "the same requests all queued at once, 4 workers"},
            "peak_running": st["peak_running"], "setup_s": round(gen_s, 1)}
    for rs in pool:
        rs.close()
    return line


def run_serve(args):
    print(json.dumps(serve_record(args.scale, args.requests)), flush=True)


# ------------------------------------------------------------- large instance
LARGE_BUDGET = 180 * 10**9


def large_recipe():
    import synth
    return synth.Recipe("metagenome-500-genomes-15Gbases", seed=55, n_genomes=500, genome_len_min=1_000_000,
                        genome_len_max=5_000_000, abundance_sigma=1.5, n_reads=100_000_000, subst_rate=0.01,
                        err_qual_lo=2, err_qual_hi=12, n_rate=1e-4)


def run_large(args):
    """The 15-Gbase, 500-genome instance at k = 55 within 180 GB of device
    memory (readset included): with the Bloom gate (k-mers seen once kept out
    of the counting pass) and without it, each after one warm-up query.  The
    survivors go straight to page-locked host arrays as the leaves find them
    (kmer_analysis_query_into with KMER_HOST), so that the device memory holds
    the reads, the records and the filters only."""
    import torch

    import synth
    import paper_1809_07014_gb300 as pkg

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    r = large_recipe()
    if args.scale != 1.0:
        r = r.scaled(max(1, int(r.n_reads * args.scale)))
    t0 = time.perf_counter()
    s = synth.generate(r)
    rs = pkg.ReadSet(s.bases, s.quals, s.offsets, stream=stream)
    n_bases = s.n_bases
    del s
    gen_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    # the packed readset counts against the 180 GB: 16 bytes per 32-base block,
    # and the base and block offsets (8 bytes each per read)
    n_reads = r.n_reads
    rs_bytes = 16 * (n_bases // 32 + n_reads) + 16 * (n_reads + 1)
    budget = LARGE_BUDGET - rs_bytes
    cap = int(0.06 * n_bases) + 4096  # survivors: about 0.81 G at this size
    t0 = time.perf_counter()
    keys = torch.empty((cap, 2), dtype=torch.int64).pin_memory()
    cnt = torch.empty(cap, dtype=torch.int32).pin_memory()
    ext = torch.empty((cap, 8), dtype=torch.int32).pin_memory()
    cls = torch.empty((cap, 2), dtype=torch.uint8).pin_memory()
    pin_s = time.perf_counter() - t0
    out = {}
    for name, flags in (("gated", pkg.KMER_FLAG_BLOOM_GATE), ("ungated", 0)):
        ka = pkg.KmerAnalysis(55, stream=stream, memory_budget=budget, flags=flags | pkg.KMER_FLAG_PROFILE)
        runs = []
        for i in range(2):
            ka.reset()
            ka.submit(rs)
            torch.cuda.synchronize()
            free_b, total_b = torch.cuda.mem_get_info()
            print(f"large: {name} query {i}: device free {free_b / 1e9:.1f} of {total_b / 1e9:.1f} GB",
                  file=sys.stderr, flush=True)
            t1 = time.perf_counter()
            v = pkg.kmer_analysis_query_into(ka.handle, keys.data_ptr(), cnt.data_ptr(), ext.data_ptr(),
                                             cls.data_ptr(), cap, pkg.KMER_HOST)
            torch.cuda.synchronize()
            runs.append(time.perf_counter() - t1)
            st = ka.stats()
            print(f"large: {name} query {i}: {runs[-1]:.3f} s, passes {st['passes']}, waves {st['l2_waves']}, "
                  f"records {st['records_emitted']}, device bytes {st['device_bytes']}, gate first {st['gate_first']} "
                  f"twice {st['gate_twice']}", file=sys.stderr, flush=True)
        out[name] = {"s": round(runs[-1], 4), "first_query_s": round(runs[0], 4),
                     "k-mers/s": int(v.windows) / runs[-1], "windows": int(v.windows),
                     "distinct": int(v.distinct), "survivors": int(v.n), "passes": st["passes"],
                     "l2_waves": st["l2_waves"], "records_emitted": st["records_emitted"],
                     "device_bytes_analysis": st["device_bytes"],
                     "gate_first": st["gate_first"], "gate_twice": st["gate_twice"],
                     "stages_ms": {k: round(st[k], 2) for k in ("ms_gate", "ms_scatter", "ms_repart", "ms_leaf",
                                                                 "ms_fallback")}}
        ka.close()
    line = {"metric": METRIC, "value": out["gated"]["k-mers/s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": 1e3 * out["gated"]["s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"one instance: {n_bases / 1e9:.1f} Gbases of 150 bp reads from 500 genomes "
                                   f"(log-normal abundance, 1% substitutions), k=55",
                       "budget_bytes": LARGE_BUDGET, "readset_bytes": int(rs_bytes),
                       "analysis_budget_bytes": int(budget)},
            "gated": out["gated"], "ungated": out["ungated"], "setup_s": round(gen_s, 1),
            "pinned_output_bytes": int(cap * (16 + 4 + 32 + 2)), "pin_s": round(pin_s, 1)}
    print(json.dumps(line), flush=True)
    rs.close()


# ------------------------------------------------------------- multi-k
def multik_record(steps: int, warmup: int) -> dict:
    """The single-genome reads (20 000 x 150 bp) resident on the device,
    analysed at k = 21, 33, 55, 77, 99 (Algorithm 1's k loop): as five
    regular queries in sequence, and as one batch of five jobs (one CUDA graph
    per wave, one launch per stage and key width)."""
    import torch

    import synth
    import paper_1809_07014_gb300 as pkg

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    s = synth.generate(synth.SINGLE_GENOME)
    rs = pkg.ReadSet(s.bases, s.quals, s.offsets, stream=stream)
    ks = [21, 33, 55, 77, 99]
    handles = {k: pkg.KmerAnalysis(k, stream=stream) for k in ks}
    cold = {}
    for k in ks:  # warm-up: allocations and learned sizing; the first query of a handle is timed
        for i in range(max(3, warmup)):
            torch.cuda.synchronize()
            tw = time.perf_counter()
            handles[k].reset(); handles[k].submit(rs); handles[k].query()
            if i == 0:
                cold[k] = round(1e3 * (time.perf_counter() - tw), 3)
    torch.cuda.synchronize()
    per_k, windows = {}, 0
    t0 = time.perf_counter()
    for _ in range(steps):
        for k in ks:
            t1 = time.perf_counter()
            ka = handles[k]
            ka.reset(); ka.submit(rs)
            v = ka.query()
            per_k.setdefault(k, []).append(time.perf_counter() - t1)
            windows += int(v.windows)
    dt = time.perf_counter() - t0
    for ka in handles.values():
        ka.close()
    # the same five analyses as one batch
    b = pkg.Batch([(rs, {"k": k}) for k in ks], stream=stream)
    for _ in range(max(3, warmup)):
        b.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        b.run()
    torch.cuda.synchronize()
    dtb = time.perf_counter() - t0
    bst = b.stats()
    b.close()
    line = {"metric": METRIC, "value": windows / dtb, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": 1e3 * dtb / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "multi-k on the single-genome reads: 20 000 x 150 bp from a 100 kbp genome, "
                                   "resident, k = 21, 33, 55, 77, 99 (a step = the five analyses)",
                       "bases": int(rs.n_bases), "l2": "inputs fit the 129 MB L2"},
            "batch": {"ms_per_round": round(1e3 * dtb / steps, 3), "graph_launches": bst["graph_launches"],
                      "waves": bst["waves"]},
            "sequential": {"value": windows / dt, "ms_per_round": round(1e3 * dt / steps, 3),
                           "per_k_ms": {k: round(1e3 * statistics.median(v), 3) for k, v in per_k.items()},
                           "cold_per_k_ms": cold}}
    rs.close()
    return line


def run_multik(args):
    print(json.dumps(multik_record(args.steps, args.warmup)), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "multik":
        run_multik(args)
    elif args.mode == "large":
        run_large(args)
    elif args.mode == "assembly":
        run_assembly(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
