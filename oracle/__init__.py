"""CPU oracle for k-mer analysis -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library never does, and it shares no code
with the CUDA path (its own parsing, reverse complement and classification,
no 2-bit packing).

The C++ side (``kmer_oracle.cpp``) writes the definition of Sec. II-B/II-C of
the paper out with strings and ``std::map``; see its header for the rules and
for the readings taken where the paper is silent.  Every function here is
pinned by ``tests/test_oracle_pins.py`` against brute force, closed forms,
invariants and generator ground truth.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkmer_oracle.so")
_lock = threading.Lock()
_lib = None

FORK = 4
DEAD_END = 5


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (plain -O2)."""
    src = os.path.join(_HERE, "kmer_oracle.cpp")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", tmp, src], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("min_count", ctypes.c_uint32),
                ("qual_offset", ctypes.c_int32), ("qual_threshold", ctypes.c_int32),
                ("ext_mode", ctypes.c_int32), ("t_base", ctypes.c_uint32),
                ("err_num", ctypes.c_uint32), ("err_den", ctypes.c_uint32),
                ("t_ext", ctypes.c_uint32)]


class _Result(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("keys", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("ext", ctypes.c_void_p), ("cls", ctypes.c_void_p),
                ("windows", ctypes.c_uint64), ("distinct", ctypes.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.oracle_kmer_analysis.argtypes = [vp, vp, vp, ctypes.c_uint64, ctypes.POINTER(_Params),
                                                 ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_Result)]
            lib.oracle_kmer_analysis.restype = ctypes.c_int
            lib.oracle_kmer_analysis_threads.argtypes = [vp, vp, vp, ctypes.c_uint64, ctypes.POINTER(_Params),
                                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                         ctypes.c_uint32, ctypes.POINTER(_Result)]
            lib.oracle_kmer_analysis_threads.restype = ctypes.c_int
            lib.oracle_merge_contigs.argtypes = [vp, vp, vp, ctypes.c_uint64, ctypes.POINTER(_Params), vp, vp,
                                                 ctypes.c_uint64, ctypes.POINTER(_Result)]
            lib.oracle_merge_contigs.restype = ctypes.c_int
            lib.oracle_traverse.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_traverse.restype = ctypes.c_int
            lib.oracle_free_contigs.argtypes = [vp, vp]
            lib.oracle_free_contigs.restype = None
            lib.oracle_free.argtypes = [ctypes.POINTER(_Result)]
            lib.oracle_free.restype = None
            lib.oracle_fnv1a.argtypes = [ctypes.c_char_p, ctypes.c_uint64]
            lib.oracle_fnv1a.restype = ctypes.c_uint64
            lib.oracle_count_keys.argtypes = [vp, vp, vp, ctypes.c_uint64, ctypes.POINTER(_Params), vp,
                                              ctypes.c_uint64, vp, vp]
            lib.oracle_count_keys.restype = ctypes.c_int
            lib.oracle_classify.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(_Params), vp]
            lib.oracle_classify.restype = None
            _lib = lib
    return _lib


@dataclass(frozen=True)
class Params:
    """Parameters of k-mer analysis as the paper states them.

    k: k-mer length.  min_count: keep k-mers seen at least this often (the
    paper's "more than epsilon", Sec. II-B).  qual_threshold: Phred at or
    above which an extension base counts.  ext_mode 0: depth adaptive
    t_hq = max(t_base, e*d) with e = err_num/err_den (Sec. II-C); ext_mode 1:
    static count threshold t_ext (Sec. II-B).
    """
    k: int
    min_count: int = 2
    qual_offset: int = 33
    qual_threshold: int = 20
    ext_mode: int = 0
    t_base: int = 2
    err_num: int = 1
    err_den: int = 10
    t_ext: int = 2

    def _c(self) -> _Params:
        return _Params(self.k, self.min_count, self.qual_offset, self.qual_threshold, self.ext_mode,
                       self.t_base, self.err_num, self.err_den, self.t_ext)


@dataclass
class Result:
    keys: np.ndarray     # (n,) bytes objects dtype S{k}, ascending
    count: np.ndarray    # (n,) uint64
    ext: np.ndarray      # (n, 8) uint64: left A,C,G,T, right A,C,G,T
    cls: np.ndarray      # (n, 2) uint8
    windows: int         # valid windows counted
    distinct: int        # distinct canonical k-mers before filtering

    def __len__(self) -> int:
        return len(self.count)


def _as_u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    return np.ascontiguousarray(a, dtype=np.uint8)


def _inputs(bases, quals, offsets):
    b = _as_u8(bases)
    q = _as_u8(quals)
    o = np.ascontiguousarray(offsets, dtype=np.uint64)
    n_reads = len(o) - 1
    if n_reads < 0 or (n_reads and int(o[-1]) > len(b)) or len(q) < len(b):
        raise ValueError("offsets do not match the base/quality buffers")
    return b, q, o, n_reads


def _collect(lib, res, rc, k) -> Result:
    if rc:
        lib.oracle_free(ctypes.byref(res))
        raise ValueError(f"oracle rejected its arguments (status {rc})")
    try:
        n = int(res.n)
        keys = np.frombuffer(ctypes.string_at(res.keys, n * k), dtype=f"S{k}").copy() if n else \
            np.empty(0, dtype=f"S{k}")
        count = np.frombuffer(ctypes.string_at(res.count, 8 * n), dtype=np.uint64).copy()
        ext = np.frombuffer(ctypes.string_at(res.ext, 64 * n), dtype=np.uint64).reshape(n, 8).copy()
        cls = np.frombuffer(ctypes.string_at(res.cls, 2 * n), dtype=np.uint8).reshape(n, 2).copy()
        return Result(keys, count, ext, cls, int(res.windows), int(res.distinct))
    finally:
        lib.oracle_free(ctypes.byref(res))


def run(bases, quals, offsets, params: Params, shard: int = 0, n_shards: int = 1) -> Result:
    """Run the oracle on reads given in the flat layout (bases, quals, offsets)."""
    lib = _load()
    b, q, o, n_reads = _inputs(bases, quals, offsets)
    res = _Result()
    cp = params._c()
    rc = lib.oracle_kmer_analysis(ctypes.c_void_p(b.ctypes.data if len(b) else 0),
                                  ctypes.c_void_p(q.ctypes.data if len(q) else 0),
                                  ctypes.c_void_p(o.ctypes.data), n_reads, ctypes.byref(cp),
                                  shard, n_shards, ctypes.byref(res))
    return _collect(lib, res, rc, params.k)


def run_threads(bases, quals, offsets, params: Params, shard_lo: int = 0, shard_hi: int = 1, n_shards: int = 1,
                threads: int = 1) -> Result:
    """The keys of shards [shard_lo, shard_hi) of n_shards (all keys with the
    defaults), the reads split into `threads` ranges counted in parallel and
    the partial maps summed before the filter (one result, ascending)."""
    lib = _load()
    b, q, o, n_reads = _inputs(bases, quals, offsets)
    res = _Result()
    cp = params._c()
    rc = lib.oracle_kmer_analysis_threads(ctypes.c_void_p(b.ctypes.data if len(b) else 0),
                                          ctypes.c_void_p(q.ctypes.data if len(q) else 0),
                                          ctypes.c_void_p(o.ctypes.data), n_reads, ctypes.byref(cp),
                                          shard_lo, shard_hi, n_shards, max(1, threads), ctypes.byref(res))
    return _collect(lib, res, rc, params.k)


def merge_contigs(bases, quals, offsets, params: Params, contigs, contig_offsets) -> Result:
    """Merge of Algorithm 1: the reads' k-mer set (`run`) with the k-mers of the
    contigs (bytes, offsets), k-mers in both kept once with the reads' record,
    contig-only k-mers added with count 0 and the classes of their contig
    neighbours (see kmer_oracle.cpp)."""
    lib = _load()
    b, q, o, n_reads = _inputs(bases, quals, offsets)
    c = _as_u8(contigs)
    co = np.ascontiguousarray(contig_offsets, dtype=np.uint64)
    n_contigs = len(co) - 1
    if n_contigs < 0 or (n_contigs and int(co[-1]) > len(c)):
        raise ValueError("contig offsets do not match the contig buffer")
    res = _Result()
    cp = params._c()
    rc = lib.oracle_merge_contigs(ctypes.c_void_p(b.ctypes.data if len(b) else 0),
                                  ctypes.c_void_p(q.ctypes.data if len(q) else 0),
                                  ctypes.c_void_p(o.ctypes.data), n_reads, ctypes.byref(cp),
                                  ctypes.c_void_p(c.ctypes.data if len(c) else 0), ctypes.c_void_p(co.ctypes.data),
                                  n_contigs, ctypes.byref(res))
    return _collect(lib, res, rc, params.k)


def traverse(keys: np.ndarray, cls: np.ndarray) -> list[bytes]:
    """De Bruijn graph traversal (Sec. II-C) over a k-mer set (keys: S{k}
    strings, cls: (n, 2) classes): the contigs, each the smaller of itself and
    its reverse complement, in ascending order (see kmer_oracle.cpp)."""
    lib = _load()
    keys = np.ascontiguousarray(keys)
    k = keys.dtype.itemsize
    cls = np.ascontiguousarray(cls, dtype=np.uint8)
    n = len(keys)
    c_ptr, o_ptr, nc = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_uint64()
    rc = lib.oracle_traverse(ctypes.c_void_p(keys.ctypes.data if n else 0), ctypes.c_void_p(cls.ctypes.data if n else 0),
                             n, k, ctypes.byref(c_ptr), ctypes.byref(o_ptr), ctypes.byref(nc))
    if rc:
        raise ValueError(f"oracle_traverse rejected its arguments (status {rc})")
    try:
        m = int(nc.value)
        offs = np.frombuffer(ctypes.string_at(o_ptr, 8 * (m + 1)), dtype=np.uint64)
        data = ctypes.string_at(c_ptr, int(offs[-1])) if m else b""
        return [data[int(offs[i]):int(offs[i + 1])] for i in range(m)]
    finally:
        lib.oracle_free_contigs(c_ptr, o_ptr)


def host_threads() -> int:
    """Cores this process may run on (all host cores unless restricted)."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def run_reads(reads, params: Params) -> Result:
    """Convenience: reads as a list of (bases, quals) byte strings (quals already offset)."""
    bases = b"".join(r[0] for r in reads)
    quals = b"".join(r[1] for r in reads)
    offsets = np.zeros(len(reads) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([len(r[0]) for r in reads], dtype=np.uint64)
    return run(bases, quals, offsets, params)


def run_shards(bases, quals, offsets, params: Params, shards, n_shards: int, threads: int) -> list[Result]:
    """Run several shards in parallel threads (the C call releases the GIL)."""
    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        return list(ex.map(lambda s: run(bases, quals, offsets, params, s, n_shards), shards))


def fnv1a(key: bytes) -> int:
    """The oracle's shard hash (FNV-1a, 64 bit) of one key string."""
    return int(_load().oracle_fnv1a(key, len(key)))


def count_keys(bases, quals, offsets, params: Params, keys: np.ndarray, threads: int = 1):
    """The definition restricted to the canonical keys `keys` (dtype S{k}):
    returns count (n,), ext (n, 8) and cls (n, 2) over all reads.  The reads
    are split into `threads` contiguous ranges counted in parallel and summed."""
    lib = _load()
    b = _as_u8(bases)
    q = _as_u8(quals)
    o = np.ascontiguousarray(offsets, dtype=np.uint64)
    n_reads = len(o) - 1
    keys = np.ascontiguousarray(keys, dtype=f"S{params.k}")
    n = len(keys)
    cp = params._c()
    cuts = np.linspace(0, n_reads, max(1, threads) + 1).astype(np.int64)
    parts = []

    def work(i):
        a, e = int(cuts[i]), int(cuts[i + 1])
        cnt = np.zeros(n, dtype=np.uint64)
        ext = np.zeros((n, 8), dtype=np.uint64)
        sub = np.ascontiguousarray(o[a:e + 1])
        rc = lib.oracle_count_keys(ctypes.c_void_p(b.ctypes.data), ctypes.c_void_p(q.ctypes.data),
                                   ctypes.c_void_p(sub.ctypes.data), e - a, ctypes.byref(cp),
                                   ctypes.c_void_p(keys.ctypes.data), n, ctypes.c_void_p(cnt.ctypes.data),
                                   ctypes.c_void_p(ext.ctypes.data))
        if rc:
            raise ValueError("oracle_count_keys rejected its arguments")
        return cnt, ext

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        parts = list(ex.map(work, range(len(cuts) - 1)))
    count = sum(p[0] for p in parts)
    ext = sum(p[1] for p in parts)
    cls = np.zeros((n, 2), dtype=np.uint8)
    for i in range(n):
        e8 = np.ascontiguousarray(ext[i])
        out = np.zeros(2, dtype=np.uint8)
        lib.oracle_classify(ctypes.c_void_p(e8.ctypes.data), int(count[i]), ctypes.byref(cp),
                            ctypes.c_void_p(out.ctypes.data))
        cls[i] = out
    return count, ext, cls
