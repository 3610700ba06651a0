"""Autotuner for the method and partition geometry of k-mer analysis.

The library sizes its partitions from the expected number of distinct
k-mers: how many leaves (shared-memory tables) a job is split into, and how
the partition bits are split between the scatter (level 1) and the
repartition (level 2).  Both trade kernel costs against each other (more
leaves = emptier tables but more per-leaf overhead; a wider level 1 = longer
scatter flushes, a wider level 2 = shorter repartition runs), and the best
point depends on the key width and the data.

The method is chosen first: the partitioned variant, the same with the
Bloom gate (k-mers seen once kept out of the counting pass: one more pass
over the reads against fewer records to partition and count), or one HBM
table updated by atomics.  Which wins depends on how many k-mers are seen
once and on memory.

``autotune`` measures the candidates on a sample readset with the
library's own stage timers (CUDA events on the analysis stream) and returns
a ``Tuning``: the measured distinct/window and survivor/window ratios plus
the winning method, "distinct keys per leaf" and level-1 share.
``Tuning.params`` turns that into per-job parameters (variant, flags,
distinct_hint, leaf_bits, l1_bits, survivors_hint) for a job of any size.
``TuningCache`` keeps tunings per (key width, size class) in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import asdict, dataclass

from . import KMER_FLAG_BLOOM_GATE, KMER_FLAG_PROFILE, KMER_VARIANT_HBM_TABLE, KmerAnalysis, ReadSet

METHODS = {"partitioned": {}, "gate": {"flags": KMER_FLAG_BLOOM_GATE},
           "hbm_table": {"variant": KMER_VARIANT_HBM_TABLE}}


@dataclass
class Tuning:
    k: int
    words: int
    windows: int
    distinct_ratio: float      # distinct canonical k-mers / windows on the sample
    survivor_ratio: float      # survivors / windows on the sample
    keys_per_leaf: float       # best expected distinct keys per leaf
    l1_shift: int              # level-1 bits relative to floor(levels / 2)
    ms_best: float
    ms_default: float
    method: str = "partitioned"                     # a key of METHODS
    method_ms: dict | None = None                   # measured time of every method tried

    def params(self, windows: int, **base) -> dict:
        """Parameters for a job of `windows` windows (a kmer_batch job dict)."""
        distinct = max(1, int(self.distinct_ratio * windows))
        leaf_bits = max(1, math.ceil(math.log2(max(2.0, distinct / self.keys_per_leaf))))
        leaf_bits = min(22, leaf_bits)
        l1 = 0
        if leaf_bits > 11:
            l1 = max(1, min(11, leaf_bits // 2 + self.l1_shift, leaf_bits - 1))
            if leaf_bits - l1 > 11:
                l1 = leaf_bits - 11
        out = dict(base)
        out.update(k=self.k, distinct_hint=int(distinct * 1.15) + 1, leaf_bits=leaf_bits, l1_bits=l1,
                   survivors_hint=int(self.survivor_ratio * windows * 1.1) + 1024)
        return out

    def method_params(self) -> dict:
        """Parameters of the chosen method (variant, flags) for a single analysis."""
        return dict(METHODS.get(self.method, {}))


def _stage_ms(st: dict) -> float:
    return st["ms_gate"] + st["ms_scatter"] + st["ms_repart"] + st["ms_leaf"] + st["ms_fallback"]


def _run(rs: ReadSet, k: int, reps: int, stream, **params) -> tuple[float, dict]:
    flags = params.pop("flags", 0) | KMER_FLAG_PROFILE
    ka = KmerAnalysis(k, stream=stream, flags=flags, **params)
    best, st = float("inf"), None
    for _ in range(reps + 1):  # the first query also teaches the handle its distinct ratio
        ka.reset()
        ka.submit(rs)
        ka.query()
        s = ka.stats()
        t = _stage_ms(s)
        if st is not None:
            best = min(best, t)
        st = s
    ka.close()
    return best, st


def autotune(rs: ReadSet, k: int, reps: int = 2, stream=None, keys_per_leaf=(0.3, 0.4, 0.5, 0.6),
             l1_shifts=(-1, 0), methods=("partitioned", "gate", "hbm_table")) -> Tuning:
    """Time the methods, then candidate geometries of the partitioned ones, for
    k on readset `rs`; return the fastest.  The gate needs min_count >= 2 (the
    default)."""
    ms_default, st = _run(rs, k, reps, stream)
    windows, distinct, surv = st["windows"], st["distinct"], st["survivors"]
    method_ms = {"partitioned": ms_default}
    for m in methods:
        if m != "partitioned":
            method_ms[m], _ = _run(rs, k, reps, stream, **METHODS[m])
    method = min(method_ms, key=method_ms.get)
    slots = st["leaf_table_slots"]
    best = (method_ms[method] if method != "hbm_table" else ms_default, 0.6, 0)
    if windows:
        for frac in keys_per_leaf:
            per_leaf = frac * slots
            leaf_bits = min(22, max(1, math.ceil(math.log2(max(2.0, distinct / per_leaf)))))
            for shift in (l1_shifts if leaf_bits > 11 else (0,)):
                l1 = 0
                if leaf_bits > 11:
                    l1 = max(1, min(11, leaf_bits // 2 + shift, leaf_bits - 1))
                    if leaf_bits - l1 > 11:
                        continue
                extra = METHODS[method] if method != "hbm_table" else {}
                ms, _ = _run(rs, k, reps, stream, leaf_bits=leaf_bits, l1_bits=l1,
                             distinct_hint=int(distinct * 1.15) + 1, **extra)
                if ms < best[0]:
                    best = (ms, per_leaf, shift)
    W = (2 * k + 63) // 64
    return Tuning(k=k, words=W, windows=windows, distinct_ratio=distinct / max(1, windows),
                  survivor_ratio=surv / max(1, windows), keys_per_leaf=best[1] if best[1] > 1 else 0.6 * slots,
                  l1_shift=best[2], ms_best=min(best[0], method_ms[method]), ms_default=ms_default, method=method,
                  method_ms={m: round(v, 3) for m, v in method_ms.items()})


class TuningCache:
    """Tunings keyed by (k, size class = log2 of the windows), in a JSON file."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.entries: dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    @staticmethod
    def _key(k: int, windows: int) -> str:
        return f"{k}:{int(math.log2(max(2, windows)))}"

    def get(self, k: int, windows: int) -> Tuning | None:
        """The tuning of this k with the nearest size class, if any."""
        best, dist = None, None
        want = int(math.log2(max(2, windows)))
        for key, v in self.entries.items():
            kk, cls = key.split(":")
            if int(kk) != k:
                continue
            d = abs(int(cls) - want)
            if dist is None or d < dist:
                best, dist = v, d
        return Tuning(**best) if best else None

    def put(self, t: Tuning) -> None:
        self.entries[self._key(t.k, t.windows)] = asdict(t)
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
