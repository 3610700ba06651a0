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
ORACLE_SAMPLE_READS = 60_000  # cpu_baseline sample: about 10-20 s of single-threaded oracle work
REF_STEP_READS = 20_000       # reference arm: reads per timed step (a few seconds each)


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
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def load_peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_traffic(name: str, src: str):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, or None
    when the summary is missing or the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_bytes = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.e+]+)", text)
    if not m_sha or not m_bytes:
        return None
    cur = hashlib.sha256(open(os.path.join(ROOT, "paper_1809_07014_gb300", "csrc", src), "rb").read()).hexdigest()
    return float(m_bytes.group(1)) if cur == m_sha.group(1) else None


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
    """Oracle (as it stands, one thread) on the first n_reads reads: windows/s."""
    import numpy as np
    import oracle
    n_reads = min(n_reads, rs.n_reads)
    end = int(rs.offsets[n_reads])
    t0 = time.perf_counter()
    res = oracle.run(rs.bases[:end], rs.quals[:end], rs.offsets[:n_reads + 1], oracle.Params(k=k))
    dt = time.perf_counter() - t0
    return res.windows / dt, dt, res.windows, n_reads


def config_of(args, recipe, n_bases):
    return {"workload": f"synthetic metagenome, {recipe.n_genomes} genomes, {n_bases / 1e9:.2f} Gbases, "
                        f"150 bp reads, k={args.k}",
            "reads": recipe.n_reads, "bases": n_bases, "read_len": 150, "k": args.k, "min_count": 2,
            "qual_threshold": 20, "variant": args.variant,
            "l2": "inputs (reads 4 GB, records >12 GB) larger than the 129 MB L2; no flush"}


# ------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return  # the oracle runs on rank 0 only
    import synth
    recipe = workload(0, args.reads)
    sample = workload(0, REF_STEP_READS)  # the first reads of the same recipe
    rs = synth.generate(sample)
    rates, wins = [], 0
    for i in range(args.warmup + args.steps):
        rate, dt, w, n = oracle_rate(rs, args.k, REF_STEP_READS)
        if i >= args.warmup:
            rates.append(rate)
            wins += w
    value = statistics.median(rates)
    desc = f"first {REF_STEP_READS} reads ({wins // max(1, args.steps)} windows) of the workload, one thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * (wins / args.steps) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": config_of(args, recipe, 150 * recipe.n_reads),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_1809_07014_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
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
    ka = pkg.KmerAnalysis(args.k, stream=stream, flags=pkg.KMER_FLAG_PROFILE, variant=variant,
                          leaf_bits=args.leaf_bits)

    def step():
        rset.pack(bases_d, quals_d, offs_d, stream=stream)
        ka.reset()
        ka.submit(rset)
        return ka.query()

    for _ in range(max(args.warmup, 3 if args.warmup else 0)):
        v = step()
    torch.cuda.synchronize()
    stage_keys = ("ms_scatter", "ms_repart", "ms_leaf", "ms_fallback", "n_scatter", "n_repart", "n_leaf",
                  "n_fallback")
    acc = {k: 0.0 for k in stage_keys}
    launches = 0
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
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
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    ms_max = ms
    tot_windows = windows
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
        w = torch.tensor([windows], device=dev, dtype=torch.float64)
        dist.all_reduce(w)
        tot_windows = int(w.item())
    value = tot_windows / (ms_max / 1e3)
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

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config_of(args, recipe, n_bases), "roofline": roofline}

    # ---- end to end through the C ABI from pinned host buffers
    if not args.no_e2e:
        b_h = torch.from_numpy(rs.bases).pin_memory()
        q_h = torch.from_numpy(rs.quals).pin_memory()
        o_h = torch.from_numpy(rs.offsets.view(np.int64)).pin_memory()
        cap = n_surv + n_surv // 8 + 1024
        keys_h = torch.empty((cap, W), dtype=torch.int64).pin_memory()
        cnt_h = torch.empty(cap, dtype=torch.int32).pin_memory()
        ext_h = torch.empty((cap, 8), dtype=torch.int32).pin_memory()
        cls_h = torch.empty((cap, 2), dtype=torch.uint8).pin_memory()
        rset_h = pkg.ReadSet(b_h, q_h, o_h, stream=stream)

        def e2e_step():
            rset_h.pack(b_h, q_h, o_h, stream=stream)
            ka.reset()
            ka.submit(rset_h)
            vv = ka.query()
            pkg.kmer_analysis_copy_results(ka.handle, keys_h.data_ptr(), cnt_h.data_ptr(), ext_h.data_ptr(),
                                           cls_h.data_ptr(), cap)
            return vv
        vv = e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.steps):
            vv = e2e_step()
            d2h += int(vv.n) * (8 * W + 4 + 32 + 2)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        h2d = 2 * n_bases + 8 * (n_reads + 1)
        line["e2e"] = {"value": tot_windows / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h // args.steps, "ms_per_step": 1e3 * dt / args.steps}
        rset_h.close()
    line["clocks"] = clocks.stop()
    line["gpu_launches"] = launches
    line["stats"] = {k: st[k] for k in ("windows", "distinct", "survivors", "passes", "l1_bits", "l2_bits",
                                        "retries", "fallback_leaves", "leaf_table_slots", "device_bytes")}

    # ---- CPU baseline: the oracle on a bounded sample, rank 0 at N = 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, dt, w, n = oracle_rate(rs, args.k, ORACLE_SAMPLE_READS)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {n} reads ({w} windows) of the same workload, "
                                          f"{dt:.1f} s on one host core ({os.cpu_count()} cores on the host)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ka.close()
    rset.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
