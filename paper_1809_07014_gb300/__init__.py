"""k-mer analysis on one GB300 GPU: Python binding of the C ABI.

Thin ctypes layer over ``libkmer_analysis.so`` (built in-tree by
``paper_1809_07014_gb300.build``).  The functions carry the C names of
``include/kmer_analysis.h`` and only marshal arguments; every step of the
computation runs in the library's CUDA kernels.  There is no CPU fallback:
if the library is missing or no GPU is present, calls raise.

Convenience wrappers (:class:`ReadSet`, :class:`KmerAnalysis`) accept numpy
arrays (host) or CUDA torch tensors (device) for the flat read layout
``bases[offsets[i]:offsets[i+1]]``.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkmer_analysis.so")

KMER_OK = 0
KMER_ERR_INVALID_ARG = -1
KMER_ERR_OOM = -2
KMER_ERR_TABLE_FULL = -3
KMER_ERR_COUNTER_OVERFLOW = -4
KMER_ERR_TIMEOUT = -5
KMER_ERR_CUDA = -6
KMER_ERR_BAD_STATE = -7
KMER_ERR_NO_DEVICE = -8
KMER_HOST, KMER_DEVICE, KMER_HOST_STAGED = 0, 1, 2
KMER_EXT_DEPTH_ADAPTIVE, KMER_EXT_STATIC = 0, 1
KMER_VARIANT_PARTITIONED, KMER_VARIANT_HBM_TABLE = 0, 1
KMER_CLS_FORK, KMER_CLS_DEAD_END = 4, 5
KMER_FLAG_PROFILE = 1
KMER_FLAG_BLOOM_GATE = 2
KMER_FLAG_SORTED_OUTPUT = 4
KMER_MAX_K = 127


class KmerError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where} failed: {code} ({detail})")
        self.code = code


class kmer_analysis_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("min_count", ctypes.c_uint32), ("qual_offset", ctypes.c_uint32),
                ("qual_threshold", ctypes.c_uint32), ("ext_mode", ctypes.c_uint32), ("t_base", ctypes.c_uint32),
                ("err_num", ctypes.c_uint32), ("err_den", ctypes.c_uint32), ("t_ext", ctypes.c_uint32),
                ("variant", ctypes.c_uint32), ("distinct_hint", ctypes.c_uint64),
                ("memory_budget", ctypes.c_uint64), ("leaf_bits", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("l1_bits", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 3)]


class kmer_result_view(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("k", ctypes.c_uint32), ("words", ctypes.c_uint32),
                ("keys", ctypes.c_void_p), ("count", ctypes.c_void_p), ("ext", ctypes.c_void_p),
                ("cls", ctypes.c_void_p), ("windows", ctypes.c_uint64), ("distinct", ctypes.c_uint64)]


class kmer_analysis_stats(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_uint64), ("distinct", ctypes.c_uint64), ("survivors", ctypes.c_uint64),
                ("records_emitted", ctypes.c_uint64), ("passes", ctypes.c_uint32), ("pass_bits", ctypes.c_uint32),
                ("l1_bits", ctypes.c_uint32), ("l2_bits", ctypes.c_uint32), ("retries", ctypes.c_uint32),
                ("fallback_leaves", ctypes.c_uint32), ("leaf_table_slots", ctypes.c_uint32),
                ("variant", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64), ("ms_total", ctypes.c_float),
                ("launches", ctypes.c_uint32), ("ms_scatter", ctypes.c_float), ("ms_repart", ctypes.c_float),
                ("ms_leaf", ctypes.c_float), ("ms_fallback", ctypes.c_float), ("n_scatter", ctypes.c_uint32),
                ("n_repart", ctypes.c_uint32), ("n_leaf", ctypes.c_uint32), ("n_fallback", ctypes.c_uint32),
                ("records_l2", ctypes.c_uint64), ("leaf_splits", ctypes.c_uint64),
                ("l2_waves", ctypes.c_uint64), ("gate_first", ctypes.c_uint64), ("gate_twice", ctypes.c_uint64),
                ("ms_gate", ctypes.c_float), ("n_gate", ctypes.c_uint32),
                ("ms_sort", ctypes.c_float), ("n_sort", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class kmer_contigs_view(ctypes.Structure):
    _fields_ = [("n_contigs", ctypes.c_uint64), ("bases", ctypes.c_uint64), ("seq", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p)]


class kmer_batch_job(ctypes.Structure):
    _fields_ = [("readset", ctypes.c_void_p), ("params", kmer_analysis_params), ("survivors_hint", ctypes.c_uint64)]


class kmer_batch_stats(ctypes.Structure):
    _fields_ = [("jobs", ctypes.c_uint32), ("waves", ctypes.c_uint32), ("graph_launches", ctypes.c_uint32),
                ("jobs_alone", ctypes.c_uint32), ("fallback_leaves", ctypes.c_uint32), ("ms_total", ctypes.c_float),
                ("jobs_repaired", ctypes.c_uint32), ("alone_level1", ctypes.c_uint32), ("alone_other", ctypes.c_uint32),
                ("replans", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class kmer_request_info(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("footprint_bytes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class kmer_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("workers", ctypes.c_uint32), ("peak_running", ctypes.c_uint32), ("pending", ctypes.c_uint32),
                ("running", ctypes.c_uint32), ("pooled", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("bytes_in_use", ctypes.c_uint64), ("budget", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


# exported symbol -> (restype, argtypes)
_vp, _u32, _u64, _int = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_SIGNATURES = {
    "kmer_analysis_default_params": (None, [ctypes.POINTER(kmer_analysis_params), _u32]),
    "kmer_readset_create": (_int, [_vp, _vp, _vp, _u64, _u32, _u32, _int, _vp, ctypes.POINTER(_vp)]),
    "kmer_readset_pack": (_int, [_vp, _vp, _vp, _vp, _u64, _int, _vp]),
    "kmer_readset_launches": (_int, [_vp, ctypes.POINTER(_u32)]),
    "kmer_readset_info": (_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "kmer_readset_destroy": (_int, [_vp]),
    "kmer_analysis_create": (_int, [ctypes.POINTER(kmer_analysis_params), _vp, ctypes.POINTER(_vp)]),
    "kmer_analysis_submit": (_int, [_vp, _vp]),
    "kmer_analysis_submit_raw": (_int, [_vp, _vp, _vp, _vp, _u64, _int]),
    "kmer_analysis_query": (_int, [_vp, ctypes.POINTER(kmer_result_view)]),
    "kmer_analysis_copy_results": (_int, [_vp, _vp, _vp, _vp, _vp, _u64]),
    "kmer_analysis_lookup": (_int, [_vp, _vp, _u64, _vp, _int]),
    "kmer_analysis_query_into": (_int, [_vp, _vp, _vp, _vp, _vp, _u64, _int, ctypes.POINTER(kmer_result_view)]),
    "kmer_analysis_merge_contigs": (_int, [_vp, _vp, _vp, _u64, _int, ctypes.POINTER(_u64),
                                           ctypes.POINTER(kmer_result_view)]),
    "kmer_analysis_traverse": (_int, [_vp, ctypes.POINTER(kmer_contigs_view)]),
    "kmer_analysis_copy_contigs": (_int, [_vp, _vp, _vp, _u64, _u64]),
    "kmer_analysis_get_stats": (_int, [_vp, ctypes.POINTER(kmer_analysis_stats)]),
    "kmer_analysis_reset": (_int, [_vp]),
    "kmer_analysis_destroy": (_int, [_vp]),
    "kmer_batch_create": (_int, [ctypes.POINTER(kmer_batch_job), _u32, _u64, _vp, ctypes.POINTER(_vp)]),
    "kmer_batch_run": (_int, [_vp]),
    "kmer_batch_result": (_int, [_vp, _u32, ctypes.POINTER(kmer_result_view)]),
    "kmer_batch_copy_results": (_int, [_vp, _u32, _vp, _vp, _vp, _vp, _u64]),
    "kmer_batch_get_stats": (_int, [_vp, ctypes.POINTER(kmer_batch_stats)]),
    "kmer_batch_destroy": (_int, [_vp]),
    "kmer_server_create": (_int, [_u64, _u32, ctypes.POINTER(_vp)]),
    "kmer_server_submit": (_int, [_vp, _vp, ctypes.POINTER(kmer_analysis_params), ctypes.POINTER(_u64)]),
    "kmer_server_poll": (_int, [_vp, _u64, ctypes.POINTER(ctypes.c_int)]),
    "kmer_server_wait": (_int, [_vp, _u64, ctypes.POINTER(kmer_result_view), ctypes.POINTER(kmer_request_info)]),
    "kmer_server_copy_results": (_int, [_vp, _u64, _vp, _vp, _vp, _vp, _u64]),
    "kmer_server_release": (_int, [_vp, _u64]),
    "kmer_server_get_stats": (_int, [_vp, ctypes.POINTER(kmer_server_stats)]),
    "kmer_server_destroy": (_int, [_vp]),
    "kmer_analysis_run_noalloc": (_int, [_vp, _vp, _vp, _u64, ctypes.POINTER(kmer_analysis_params), _vp, _vp, _vp,
                                         _vp, _u64, ctypes.POINTER(_u64), _vp]),
    "kmer_strerror": (ctypes.c_char_p, [_int]),
    "kmer_last_error_message": (ctypes.c_char_p, []),
    "kmer_version": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"{p} is missing: build the CUDA library first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(p)
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(code: int, where: str):
    if code != KMER_OK:
        lib = load_library()
        raise KmerError(code, where, lib.kmer_last_error_message().decode(errors="replace"))


# ------------------------------------------------------------ C-ABI mirrors
def kmer_analysis_default_params(k: int) -> kmer_analysis_params:
    p = kmer_analysis_params()
    load_library().kmer_analysis_default_params(ctypes.byref(p), k)
    return p


def kmer_readset_create(bases: int, quals: int, offsets: int, n_reads: int, qual_offset: int,
                        qual_threshold: int, where: int, stream: int = 0) -> int:
    out = _vp()
    _check(load_library().kmer_readset_create(bases, quals, offsets, n_reads, qual_offset, qual_threshold,
                                              where, stream or None, ctypes.byref(out)), "kmer_readset_create")
    return out.value


def kmer_readset_pack(rs: int, bases: int, quals: int, offsets: int, n_reads: int, where: int,
                      stream: int = 0) -> None:
    _check(load_library().kmer_readset_pack(rs, bases, quals, offsets, n_reads, where, stream or None),
           "kmer_readset_pack")


def kmer_readset_launches(rs: int) -> int:
    n = _u32()
    _check(load_library().kmer_readset_launches(rs, ctypes.byref(n)), "kmer_readset_launches")
    return n.value


def kmer_readset_info(rs: int) -> tuple[int, int]:
    n, b = _u64(), _u64()
    _check(load_library().kmer_readset_info(rs, ctypes.byref(n), ctypes.byref(b)), "kmer_readset_info")
    return n.value, b.value


def kmer_readset_destroy(rs: int) -> None:
    _check(load_library().kmer_readset_destroy(rs), "kmer_readset_destroy")


def kmer_analysis_create(params: kmer_analysis_params, stream: int = 0) -> int:
    out = _vp()
    _check(load_library().kmer_analysis_create(ctypes.byref(params), stream or None, ctypes.byref(out)),
           "kmer_analysis_create")
    return out.value


def kmer_analysis_submit(h: int, rs: int) -> None:
    _check(load_library().kmer_analysis_submit(h, rs), "kmer_analysis_submit")


def kmer_analysis_submit_raw(h: int, bases: int, quals: int, offsets: int, n_reads: int, where: int) -> None:
    _check(load_library().kmer_analysis_submit_raw(h, bases, quals, offsets, n_reads, where),
           "kmer_analysis_submit_raw")


def kmer_analysis_query(h: int) -> kmer_result_view:
    v = kmer_result_view()
    _check(load_library().kmer_analysis_query(h, ctypes.byref(v)), "kmer_analysis_query")
    return v


# One looked-up k-mer (kmer_record, 40 bytes).
KMER_RECORD_DTYPE = np.dtype([("count", "<u4"), ("ext", "<u4", (8,)), ("cls", "u1", (2,)), ("found", "u1"),
                              ("flipped", "u1")])
assert KMER_RECORD_DTYPE.itemsize == 40


def kmer_analysis_query_into(h: int, keys: int, count: int, ext: int, cls: int, capacity: int,
                             where: int) -> kmer_result_view:
    v = kmer_result_view()
    _check(load_library().kmer_analysis_query_into(h, keys, count, ext, cls, capacity, where, ctypes.byref(v)),
           "kmer_analysis_query_into")
    return v


def kmer_analysis_merge_contigs(h: int, contigs: int, offsets: int, n_contigs: int, where: int):
    """Merge the last query's survivors with the contigs' k-mers; returns (added, view)."""
    added = _u64()
    v = kmer_result_view()
    _check(load_library().kmer_analysis_merge_contigs(h, contigs, offsets, n_contigs, where, ctypes.byref(added),
                                                      ctypes.byref(v)), "kmer_analysis_merge_contigs")
    return added.value, v


def kmer_analysis_traverse(h: int) -> kmer_contigs_view:
    v = kmer_contigs_view()
    _check(load_library().kmer_analysis_traverse(h, ctypes.byref(v)), "kmer_analysis_traverse")
    return v


def kmer_analysis_copy_contigs(h: int, seq: int, offsets: int, seq_capacity: int, contig_capacity: int) -> None:
    _check(load_library().kmer_analysis_copy_contigs(h, seq, offsets, seq_capacity, contig_capacity),
           "kmer_analysis_copy_contigs")


def kmer_analysis_lookup(h: int, keys: int, n: int, out: int, where: int) -> None:
    _check(load_library().kmer_analysis_lookup(h, keys, n, out, where), "kmer_analysis_lookup")


def kmer_analysis_copy_results(h: int, keys: int, count: int, ext: int, cls: int, capacity: int) -> None:
    _check(load_library().kmer_analysis_copy_results(h, keys, count, ext, cls, capacity),
           "kmer_analysis_copy_results")


def kmer_analysis_get_stats(h: int) -> kmer_analysis_stats:
    s = kmer_analysis_stats()
    _check(load_library().kmer_analysis_get_stats(h, ctypes.byref(s)), "kmer_analysis_get_stats")
    return s


def kmer_analysis_reset(h: int) -> None:
    _check(load_library().kmer_analysis_reset(h), "kmer_analysis_reset")


def kmer_analysis_destroy(h: int) -> None:
    _check(load_library().kmer_analysis_destroy(h), "kmer_analysis_destroy")


def kmer_analysis_run_noalloc(bases: int, quals: int, offsets: int, n_reads: int, params: kmer_analysis_params,
                              keys: int, count: int, ext: int, cls: int, capacity: int, stream: int = 0) -> int:
    """Run the allocation-free entry point; returns the number of survivors."""
    n = _u64()
    _check(load_library().kmer_analysis_run_noalloc(bases, quals, offsets, n_reads, ctypes.byref(params), keys,
                                                    count, ext, cls, capacity, ctypes.byref(n), stream or None),
           "kmer_analysis_run_noalloc")
    return n.value


def kmer_batch_create(jobs, memory_budget: int = 0, stream: int = 0) -> int:
    arr = (kmer_batch_job * max(1, len(jobs)))(*jobs)
    out = _vp()
    _check(load_library().kmer_batch_create(arr, len(jobs), memory_budget, stream or None, ctypes.byref(out)),
           "kmer_batch_create")
    return out.value


def kmer_batch_run(b: int) -> None:
    _check(load_library().kmer_batch_run(b), "kmer_batch_run")


def kmer_batch_result(b: int, job: int) -> kmer_result_view:
    v = kmer_result_view()
    _check(load_library().kmer_batch_result(b, job, ctypes.byref(v)), "kmer_batch_result")
    return v


def kmer_batch_copy_results(b: int, job: int, keys: int, count: int, ext: int, cls: int, capacity: int) -> None:
    _check(load_library().kmer_batch_copy_results(b, job, keys, count, ext, cls, capacity),
           "kmer_batch_copy_results")


def kmer_batch_get_stats(b: int) -> kmer_batch_stats:
    st = kmer_batch_stats()
    _check(load_library().kmer_batch_get_stats(b, ctypes.byref(st)), "kmer_batch_get_stats")
    return st


def kmer_batch_destroy(b: int) -> None:
    _check(load_library().kmer_batch_destroy(b), "kmer_batch_destroy")


def kmer_server_create(memory_budget: int = 0, workers: int = 4) -> int:
    out = _vp()
    _check(load_library().kmer_server_create(memory_budget, workers, ctypes.byref(out)), "kmer_server_create")
    return out.value


def kmer_server_submit(srv: int, rs: int, params: kmer_analysis_params) -> int:
    rid = _u64()
    _check(load_library().kmer_server_submit(srv, rs, ctypes.byref(params), ctypes.byref(rid)), "kmer_server_submit")
    return rid.value


def kmer_server_poll(srv: int, rid: int) -> bool:
    d = ctypes.c_int()
    _check(load_library().kmer_server_poll(srv, rid, ctypes.byref(d)), "kmer_server_poll")
    return bool(d.value)


def kmer_server_wait(srv: int, rid: int) -> tuple[kmer_result_view, kmer_request_info]:
    v, info = kmer_result_view(), kmer_request_info()
    _check(load_library().kmer_server_wait(srv, rid, ctypes.byref(v), ctypes.byref(info)), "kmer_server_wait")
    return v, info


def kmer_server_copy_results(srv: int, rid: int, keys: int, count: int, ext: int, cls: int, capacity: int) -> None:
    _check(load_library().kmer_server_copy_results(srv, rid, keys, count, ext, cls, capacity),
           "kmer_server_copy_results")


def kmer_server_release(srv: int, rid: int) -> None:
    _check(load_library().kmer_server_release(srv, rid), "kmer_server_release")


def kmer_server_get_stats(srv: int) -> kmer_server_stats:
    st = kmer_server_stats()
    _check(load_library().kmer_server_get_stats(srv, ctypes.byref(st)), "kmer_server_get_stats")
    return st


def kmer_server_destroy(srv: int) -> None:
    _check(load_library().kmer_server_destroy(srv), "kmer_server_destroy")


def kmer_strerror(code: int) -> str:
    return load_library().kmer_strerror(code).decode()


def kmer_version() -> str:
    return load_library().kmer_version().decode()


# ------------------------------------------------------ convenience layer
def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (no copy)."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _where(a, staged: bool = False) -> int:
    if hasattr(a, "is_cuda") and a.is_cuda:
        return KMER_DEVICE
    return KMER_HOST_STAGED if staged else KMER_HOST


def _stream_of(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def make_params(k: int, **kw) -> kmer_analysis_params:
    p = kmer_analysis_default_params(k)
    for key, v in kw.items():
        if not hasattr(p, key):
            raise AttributeError(f"unknown parameter {key}")
        setattr(p, key, v)
    return p


class ReadSet:
    """Packed reads resident on the GPU (step a1)."""

    def __init__(self, bases, quals, offsets, qual_offset: int = 33, qual_threshold: int = 20, stream=None,
                 staged: bool = False):
        """staged: host reads are copied to the device by the copy engines
        (KMER_HOST_STAGED) even when page-locked, instead of read in place."""
        where = _where(bases, staged)
        if _where(quals, staged) != where or _where(offsets, staged) != where:
            raise ValueError("bases, quals and offsets must all be on the host or all on the device")
        n = len(offsets) - 1
        if n < 0:
            raise ValueError("offsets needs n_reads + 1 entries")
        self.handle = kmer_readset_create(_ptr(bases), _ptr(quals), _ptr(offsets), n, qual_offset,
                                          qual_threshold, where, _stream_of(stream))
        self.qual_offset, self.qual_threshold = qual_offset, qual_threshold

    def pack(self, bases, quals, offsets, stream=None, staged: bool = False):
        """Re-pack new reads into this readset, reusing its device buffers."""
        kmer_readset_pack(self.handle, _ptr(bases), _ptr(quals), _ptr(offsets), len(offsets) - 1,
                          _where(bases, staged), _stream_of(stream))

    @property
    def launches(self) -> int:
        return kmer_readset_launches(self.handle)

    @property
    def n_reads(self) -> int:
        return kmer_readset_info(self.handle)[0]

    @property
    def n_bases(self) -> int:
        return kmer_readset_info(self.handle)[1]

    def close(self):
        if self.handle:
            kmer_readset_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Result:
    """Survivors copied to the host.  keys: (n, W) uint64 words, word 0 most significant."""
    k: int
    keys: np.ndarray
    count: np.ndarray
    ext: np.ndarray
    cls: np.ndarray
    windows: int
    distinct: int

    def __len__(self) -> int:
        return len(self.count)


class KmerAnalysis:
    """One k-mer analysis (create / submit / query / destroy)."""

    def __init__(self, k: int, stream=None, **params):
        self.params = make_params(k, **params)
        self.handle = kmer_analysis_create(self.params, _stream_of(stream))
        self._keep = []

    def submit(self, rs: ReadSet):
        kmer_analysis_submit(self.handle, rs.handle)
        self._keep.append(rs)

    def submit_raw(self, bases, quals, offsets):
        where = _where(bases)
        kmer_analysis_submit_raw(self.handle, _ptr(bases), _ptr(quals), _ptr(offsets), len(offsets) - 1, where)

    def query(self) -> kmer_result_view:
        return kmer_analysis_query(self.handle)

    def results(self, view: kmer_result_view | None = None) -> Result:
        v = view if view is not None else self.query()
        n, W = int(v.n), int(v.words)
        keys = np.empty((n, W), dtype=np.uint64)
        count = np.empty(n, dtype=np.uint32)
        ext = np.empty((n, 8), dtype=np.uint32)
        cls = np.empty((n, 2), dtype=np.uint8)
        kmer_analysis_copy_results(self.handle, _ptr(keys), _ptr(count), _ptr(ext), _ptr(cls), n)
        return Result(int(v.k), keys, count, ext, cls, int(v.windows), int(v.distinct))

    def traverse(self) -> list[bytes]:
        """Contigs of the de Bruijn graph traversal (Sec. II-C) over the current
        k-mer set, each the smaller of itself and its reverse complement."""
        v = kmer_analysis_traverse(self.handle)
        seq = np.empty(max(1, int(v.bases)), dtype=np.uint8)
        offs = np.empty(int(v.n_contigs) + 1, dtype=np.uint64)
        kmer_analysis_copy_contigs(self.handle, _ptr(seq), _ptr(offs), int(v.bases), int(v.n_contigs))
        data = seq.tobytes()
        return [data[int(offs[i]):int(offs[i + 1])] for i in range(int(v.n_contigs))]

    def merge_contigs(self, contigs, offsets) -> Result:
        """Merge (Algorithm 1) of the last query's survivors with the k-mers of
        contigs given flat (bytes or uint8 array, offsets); returns the merged set."""
        where = _where(contigs)
        c = contigs if where == KMER_DEVICE else np.ascontiguousarray(np.frombuffer(bytes(contigs), np.uint8)
                                                                      if isinstance(contigs, (bytes, bytearray))
                                                                      else contigs, dtype=np.uint8)
        o = offsets if where == KMER_DEVICE else np.ascontiguousarray(offsets, dtype=np.uint64)
        n = len(o) - 1
        _, v = kmer_analysis_merge_contigs(self.handle, _ptr(c) if n else 0, _ptr(o), n, where)
        return self.results(v)

    def lookup(self, keys) -> np.ndarray:
        """Records (KMER_RECORD_DTYPE) of k-mers given as an (n, W) uint64 array,
        either orientation, among the survivors of the last query."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        if keys.ndim == 1:
            keys = keys.reshape(-1, 1)
        out = np.zeros(len(keys), dtype=KMER_RECORD_DTYPE)
        kmer_analysis_lookup(self.handle, _ptr(keys), len(keys), _ptr(out), KMER_HOST)
        return out

    def stats(self) -> dict:
        return kmer_analysis_get_stats(self.handle).as_dict()

    def reset(self):
        kmer_analysis_reset(self.handle)
        self._keep.clear()

    def close(self):
        if self.handle:
            kmer_analysis_destroy(self.handle)
            self.handle = 0
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



class Batch:
    """Many analyses run together (kmer_batch_*): jobs are (ReadSet, params) pairs,
    params given as keyword dicts over kmer_analysis_params fields (``k`` required)
    plus an optional ``survivors_hint``."""

    def __init__(self, jobs, memory_budget: int = 0, stream=None):
        cj = []
        self._keep = []
        for rs, kw in jobs:
            kw = dict(kw)
            hint = int(kw.pop("survivors_hint", 0))
            k = kw.pop("k")
            cj.append(kmer_batch_job(rs.handle, make_params(k, **kw), hint))
            self._keep.append(rs)
        self.n = len(cj)
        self.handle = kmer_batch_create(cj, memory_budget, _stream_of(stream))

    def run(self):
        kmer_batch_run(self.handle)

    def view(self, i: int) -> kmer_result_view:
        return kmer_batch_result(self.handle, i)

    def results(self, i: int) -> Result:
        v = self.view(i)
        n, W = int(v.n), int(v.words)
        keys = np.empty((n, W), dtype=np.uint64)
        count = np.empty(n, dtype=np.uint32)
        ext = np.empty((n, 8), dtype=np.uint32)
        cls = np.empty((n, 2), dtype=np.uint8)
        kmer_batch_copy_results(self.handle, i, _ptr(keys), _ptr(count), _ptr(ext), _ptr(cls), n)
        return Result(int(v.k), keys, count, ext, cls, int(v.windows), int(v.distinct))

    def stats(self) -> dict:
        return kmer_batch_get_stats(self.handle).as_dict()

    def close(self):
        if self.handle:
            kmer_batch_destroy(self.handle)
            self.handle = 0
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop (kmer_server_*): submit(readset, k=..., ...) from any thread,
    wait(id) for the device view and timestamps, results(id) for a host copy,
    release(id) when done."""

    def __init__(self, memory_budget: int = 0, workers: int = 4):
        self.handle = kmer_server_create(memory_budget, workers)
        self._keep = {}

    def submit(self, rs: ReadSet, k: int, **params) -> int:
        rid = kmer_server_submit(self.handle, rs.handle, make_params(k, **params))
        self._keep[rid] = rs
        return rid

    def done(self, rid: int) -> bool:
        return kmer_server_poll(self.handle, rid)

    def wait(self, rid: int):
        v, info = kmer_server_wait(self.handle, rid)
        return v, info.as_dict()

    def results(self, rid: int) -> Result:
        v, _ = self.wait(rid)
        n, W = int(v.n), int(v.words)
        keys = np.empty((n, W), dtype=np.uint64)
        count = np.empty(n, dtype=np.uint32)
        ext = np.empty((n, 8), dtype=np.uint32)
        cls = np.empty((n, 2), dtype=np.uint8)
        kmer_server_copy_results(self.handle, rid, _ptr(keys), _ptr(count), _ptr(ext), _ptr(cls), n)
        return Result(int(v.k), keys, count, ext, cls, int(v.windows), int(v.distinct))

    def release(self, rid: int):
        kmer_server_release(self.handle, rid)
        self._keep.pop(rid, None)

    def stats(self) -> dict:
        return kmer_server_get_stats(self.handle).as_dict()

    def close(self):
        if self.handle:
            kmer_server_destroy(self.handle)
            self.handle = 0
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
