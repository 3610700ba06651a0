"""Seeded synthetic metagenome reads (input recipe; no k-mer arithmetic here).

The C generator in ``synth.c`` draws genomes, read placements, substitution
errors, N bases and Phred qualities from per-item counter-based streams.  This
module compiles it on first use and wraps it with ctypes.  Named presets give
the workloads used by the tests and the benchmark; the recipe mimics the MGSim
inputs of the paper (Sec. IV-A): random genomes with log-normal abundance,
reads from both strands, uniform substitutions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libsynth.so (host C, OpenMP).  Returns its path."""
    src = os.path.join(_HERE, "synth.c")
    hdr = os.path.join(_HERE, "synth.h")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(src), os.path.getmtime(hdr)):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64), ("n_genomes", ctypes.c_uint32),
        ("genome_len_min", ctypes.c_uint64), ("genome_len_max", ctypes.c_uint64),
        ("abundance_sigma", ctypes.c_double), ("n_reads", ctypes.c_uint64),
        ("read_len_min", ctypes.c_uint32), ("read_len_max", ctypes.c_uint32),
        ("subst_rate", ctypes.c_double), ("err_qual_lo", ctypes.c_int), ("err_qual_hi", ctypes.c_int),
        ("qual_mean", ctypes.c_double), ("qual_sd", ctypes.c_double),
        ("qual_min", ctypes.c_int), ("qual_max", ctypes.c_int),
        ("n_rate", ctypes.c_double), ("n_qual", ctypes.c_int), ("qual_offset", ctypes.c_int),
        ("n_threads", ctypes.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            vp = ctypes.c_void_p
            lib.synth_genome_lengths.argtypes = [P, vp]
            lib.synth_genomes.argtypes = [P, vp, vp]
            lib.synth_read_offsets.argtypes = [P, vp]
            lib.synth_reads.argtypes = [P, vp, vp, vp, vp, vp, vp, vp, vp]
            for f in (lib.synth_genome_lengths, lib.synth_genomes, lib.synth_read_offsets, lib.synth_reads):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass(frozen=True)
class Recipe:
    """One synthetic workload.  Field meanings follow ``synth.h``."""
    name: str
    seed: int
    n_genomes: int
    genome_len_min: int
    genome_len_max: int
    abundance_sigma: float
    n_reads: int
    read_len_min: int = 150
    read_len_max: int = 150
    subst_rate: float = 0.0
    err_qual_lo: int = -1
    err_qual_hi: int = -1
    qual_mean: float = 32.0
    qual_sd: float = 5.0
    qual_min: int = 2
    qual_max: int = 41
    n_rate: float = 0.0
    n_qual: int = 2
    qual_offset: int = 33

    def scaled(self, n_reads: int, **kw) -> "Recipe":
        return replace(self, n_reads=n_reads, **kw)


@dataclass
class ReadSet:
    """Reads in the flat layout of the C-ABI: bases[offsets[i]:offsets[i+1]]."""
    bases: np.ndarray      # uint8 ASCII (A,C,G,T,N)
    quals: np.ndarray      # uint8 Phred + qual_offset
    offsets: np.ndarray    # uint64, n_reads + 1
    recipe: Recipe
    genomes: np.ndarray | None = None        # uint8 concatenated genomes
    genome_lens: np.ndarray | None = None    # uint64
    truth_genome: np.ndarray | None = None   # uint32 per read
    truth_pos: np.ndarray | None = None      # uint64 per read
    truth_strand: np.ndarray | None = None   # uint8 per read (1 = reverse complement)
    extra: dict = field(default_factory=dict)

    @property
    def n_reads(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_bases(self) -> int:
        return int(self.offsets[-1])

    def read(self, i: int) -> tuple[bytes, bytes]:
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return self.bases[a:b].tobytes(), self.quals[a:b].tobytes()


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def generate(r: Recipe, threads: int | None = None, truth: bool = False) -> ReadSet:
    """Draw the reads of recipe ``r`` (deterministic in ``r`` alone)."""
    lib = _load()
    p = _Params(r.seed, r.n_genomes, r.genome_len_min, r.genome_len_max, r.abundance_sigma,
                r.n_reads, r.read_len_min, r.read_len_max, r.subst_rate, r.err_qual_lo,
                r.err_qual_hi, r.qual_mean, r.qual_sd, r.qual_min, r.qual_max, r.n_rate,
                r.n_qual, r.qual_offset, int(threads or os.cpu_count() or 1))
    pp = ctypes.byref(p)
    lens = np.zeros(r.n_genomes, dtype=np.uint64)
    if lib.synth_genome_lengths(pp, _ptr(lens)):
        raise ValueError(f"invalid synthetic recipe {r}")
    genomes = np.empty(int(lens.sum()), dtype=np.uint8)
    lib.synth_genomes(pp, _ptr(lens), _ptr(genomes))
    offsets = np.empty(r.n_reads + 1, dtype=np.uint64)
    lib.synth_read_offsets(pp, _ptr(offsets))
    n = int(offsets[-1])
    bases = np.empty(n, dtype=np.uint8)
    quals = np.empty(n, dtype=np.uint8)
    tg = np.empty(r.n_reads, dtype=np.uint32) if truth else None
    tp = np.empty(r.n_reads, dtype=np.uint64) if truth else None
    ts = np.empty(r.n_reads, dtype=np.uint8) if truth else None
    rc = lib.synth_reads(pp, _ptr(lens), _ptr(genomes), _ptr(offsets), _ptr(bases), _ptr(quals),
                         _ptr(tg), _ptr(tp), _ptr(ts))
    if rc:
        raise RuntimeError(f"synth_reads failed ({rc})")
    return ReadSet(bases, quals, offsets, r,
                   genomes if truth else None, lens if truth else None, tg, tp, ts)


# --- workloads -------------------------------------------------------------
# Single genome: 100 kbp uniform-random genome, 20 000 reads x 150 bp (30x),
# both strands, 0.5 % substitutions, Phred ~ N(32, 5) clipped to [2, 41].
SINGLE_GENOME = Recipe("single-genome-100kbp-20k-reads", seed=1, n_genomes=1,
                       genome_len_min=100_000, genome_len_max=100_000, abundance_sigma=0.0,
                       n_reads=20_000, subst_rate=0.005)

# Synthetic metagenome: 50 genomes of 1-5 Mbp, log-normal abundance (sigma 1.5),
# 13 333 334 reads x 150 bp = 2 Gbases, 1 % substitutions whose bases get
# Phred U[2, 12], 0.01 % N bases (Phred 2).
METAGENOME_2G = Recipe("metagenome-50-genomes-2Gbases", seed=2, n_genomes=50,
                       genome_len_min=1_000_000, genome_len_max=5_000_000, abundance_sigma=1.5,
                       n_reads=13_333_334, subst_rate=0.01, err_qual_lo=2, err_qual_hi=12,
                       n_rate=1e-4)


def metagenome_sample(i: int, n_bases: int, n_genomes: int) -> Recipe:
    """One sample of the batched workload: a metagenome-style mixture of its own."""
    return Recipe(f"metagenome-sample-{i}", seed=4000 + i, n_genomes=n_genomes,
                  genome_len_min=1_000_000, genome_len_max=5_000_000, abundance_sigma=1.5,
                  n_reads=max(1, n_bases // 150), subst_rate=0.01, err_qual_lo=2,
                  err_qual_hi=12, n_rate=1e-4)
