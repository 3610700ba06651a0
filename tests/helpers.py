"""Test-side helpers: compare the library's output with the oracle's.

Keys from the library are 2-bit words (word 0 most significant); the oracle
returns strings.  These helpers convert and sort both sides; they share no
code with either implementation.
"""
import numpy as np

LUT = np.frombuffer(b"ACGT", dtype=np.uint8)


def decode_keys(keys: np.ndarray, k: int) -> np.ndarray:
    """(n, W) uint64 words -> (n,) byte strings of length k."""
    n, W = keys.shape
    hb = 2 * k - 64 * (W - 1)
    out = np.empty((n, k), dtype=np.uint8)
    pos = 0
    for w in range(W):
        bits = hb if w == 0 else 64
        for j in range(bits // 2):
            shift = np.uint64(bits - 2 - 2 * j)
            out[:, pos] = LUT[((keys[:, w] >> shift) & np.uint64(3)).astype(np.intp)]
            pos += 1
    return out.reshape(n * k).view(f"S{k}") if n else np.empty(0, dtype=f"S{k}")


def sorted_gpu(res):
    """GPU result -> (keys as strings, count, ext, cls) sorted by key."""
    keys = decode_keys(res.keys, res.k)
    order = np.argsort(keys, kind="stable")
    return keys[order], res.count[order].astype(np.uint64), res.ext[order].astype(np.uint64), res.cls[order]


def assert_same(gpu_res, orc_res, label=""):
    gk, gc, ge, gcl = sorted_gpu(gpu_res)
    assert len(gk) == len(orc_res.keys), f"{label}: {len(gk)} survivors on the GPU, {len(orc_res.keys)} in the oracle"
    if len(gk) > 1:
        assert (gk[1:] > gk[:-1]).all(), f"{label}: duplicate keys in the GPU output"
    bad = np.nonzero(gk != orc_res.keys)[0]
    assert bad.size == 0, f"{label}: key mismatch at {bad[:5]}: {gk[bad[:3]]} vs {orc_res.keys[bad[:3]]}"
    bad = np.nonzero(gc != orc_res.count)[0]
    assert bad.size == 0, f"{label}: count mismatch at {gk[bad[:3]]}: {gc[bad[:3]]} vs {orc_res.count[bad[:3]]}"
    bad = np.nonzero((ge != orc_res.ext).any(1))[0]
    assert bad.size == 0, f"{label}: ext mismatch at {gk[bad[:3]]}: {ge[bad[:3]]} vs {orc_res.ext[bad[:3]]}"
    bad = np.nonzero((gcl != orc_res.cls).any(1))[0]
    assert bad.size == 0, f"{label}: class mismatch at {gk[bad[:3]]}: {gcl[bad[:3]]} vs {orc_res.cls[bad[:3]]}"
    assert gpu_res.windows == orc_res.windows, f"{label}: windows {gpu_res.windows} vs {orc_res.windows}"
    assert gpu_res.distinct == orc_res.distinct, f"{label}: distinct {gpu_res.distinct} vs {orc_res.distinct}"


def fnv1a_keys(keys: np.ndarray) -> np.ndarray:
    """FNV-1a 64 of each fixed-length key string (vectorised)."""
    k = keys.dtype.itemsize
    b = keys.view(np.uint8).reshape(len(keys), k)
    h = np.full(len(keys), 14695981039346656037, dtype=np.uint64)
    prime = np.uint64(1099511628211)
    with np.errstate(over="ignore"):
        for i in range(k):
            h ^= b[:, i].astype(np.uint64)
            h *= prime
    return h
