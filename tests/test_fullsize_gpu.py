"""Full-size check on the 2-Gbase metagenome at k = 31, in the benchmark's
launch configuration (default parameters, reads resident on the device).

The oracle cannot count all 1.6 G windows in a test, so:
  * properties that hold at any size are checked on every survivor (unique,
    canonical keys; count >= min_count; tallies <= count; classes follow the
    rule) and the total window count is checked against an independent
    count of windows without N;
  * sampled outputs are computed one by one by the oracle's key-set mode over
    all reads: 3000 random survivors (exact count, tallies, classes) and 3000
    canonical k-mers taken from random read windows (present on the GPU iff
    their oracle count reaches min_count, with equal values).
"""
import os

import numpy as np
import pytest

import oracle
import synth
import paper_1809_07014_gb300 as pkg
from tests.helpers import decode_keys

pytestmark = pytest.mark.gpu
K = 31
COMP = bytes.maketrans(b"ACGT", b"TGCA")


def encode(keys: np.ndarray) -> np.ndarray:
    """S31 strings -> packed uint64 (2 bits per base, first base most significant)."""
    codes = np.frombuffer(keys.tobytes(), dtype=np.uint8).reshape(len(keys), K)
    lut = np.zeros(256, dtype=np.uint64)
    lut[ord("C")], lut[ord("G")], lut[ord("T")] = 1, 2, 3
    v = np.zeros(len(keys), dtype=np.uint64)
    for j in range(K):
        v = (v << np.uint64(2)) | lut[codes[:, j]]
    return v


def revcomp_packed(x: np.ndarray) -> np.ndarray:
    y = ~x & np.uint64((1 << 62) - 1)
    out = np.zeros_like(y)
    for j in range(K):  # base j (from the right) goes to position K-1-j
        out |= ((y >> np.uint64(2 * j)) & np.uint64(3)) << np.uint64(2 * (K - 1 - j))
    return out


def classify_rule(ext4: np.ndarray, count: np.ndarray, p) -> np.ndarray:
    """Depth-adaptive rule written over arrays (property check at full size)."""
    best = ext4.max(1)
    m = ext4.argmax(1)
    ties = (ext4 == best[:, None]).sum(1)
    alt = ext4.sum(1) - best
    lim = np.maximum(np.uint64(p.t_base * p.err_den), np.uint64(p.err_num) * count)
    out = np.where(alt * np.uint64(p.err_den) <= lim, m, 4).astype(np.uint8)
    out[ties > 1] = 4
    out[best == 0] = 5
    return out


def valid_windows(rs) -> int:
    lens = np.diff(rs.offsets).astype(np.int64)
    total = int(np.maximum(lens - K + 1, 0).sum())
    npos = np.nonzero(rs.bases == ord("N"))[0].astype(np.int64)
    if npos.size == 0:
        return total
    read = np.searchsorted(rs.offsets.astype(np.int64), npos, side="right") - 1
    lost = 0
    start = rs.offsets.astype(np.int64)
    i = 0
    while i < npos.size:  # windows of one read that contain at least one N
        r = read[i]
        j = i
        covered = -1
        L = int(lens[r])
        while j < npos.size and read[j] == r:
            p = int(npos[j] - start[r])
            lo, hi = max(p - K + 1, 0, covered + 1), min(p, L - K)
            if hi >= lo:
                lost += hi - lo + 1
                covered = hi
            j += 1
        i = j
    return total - lost


def test_metagenome_2gbases_k31(tmp_path):
    import torch
    threads = os.cpu_count() or 1
    rs = synth.generate(synth.METAGENOME_2G, threads=threads)
    dev = [torch.from_numpy(a).cuda() for a in (rs.bases, rs.quals, rs.offsets.view(np.int64))]
    stream = torch.cuda.current_stream()
    r = pkg.ReadSet(*dev, stream=stream)
    ka = pkg.KmerAnalysis(K, stream=stream)
    ka.submit(r)
    res = ka.results()
    st = ka.stats()
    ka.close()
    r.close()
    del dev
    p = oracle.Params(k=K)
    n = len(res)
    assert st["retries"] == 0 or st["retries"] <= 2
    # ---- properties of every output
    assert res.windows == valid_windows(rs)
    assert res.distinct >= n
    keys = res.keys[:, 0]
    order = np.argsort(keys)
    sk = keys[order]
    assert (sk[1:] > sk[:-1]).all(), "duplicate keys"
    assert (keys <= revcomp_packed(keys)).all(), "non-canonical key"
    assert (keys >> np.uint64(62) == 0).all()
    cnt = res.count.astype(np.uint64)
    ext = res.ext.astype(np.uint64)
    assert (cnt >= p.min_count).all()
    assert (ext[:, :4].sum(1) <= cnt).all() and (ext[:, 4:].sum(1) <= cnt).all()
    assert (classify_rule(ext[:, :4], cnt, p) == res.cls[:, 0]).all()
    assert (classify_rule(ext[:, 4:], cnt, p) == res.cls[:, 1]).all()
    # ---- sampled exact comparison with the oracle over all reads
    rng = np.random.default_rng(2026)
    pick = rng.choice(n, 3000, replace=False)
    surv_keys = decode_keys(res.keys[pick], K)
    win_keys = []
    while len(win_keys) < 3000:
        i = int(rng.integers(rs.n_reads))
        a, b = int(rs.offsets[i]), int(rs.offsets[i + 1])
        if b - a < K:
            continue
        s = int(rng.integers(b - a - K + 1))
        w = rs.bases[a + s:a + s + K].tobytes()
        if b"N" in w:
            continue
        rc = w.translate(COMP)[::-1]
        win_keys.append(min(w, rc))
    win_keys = np.array(win_keys, dtype=f"S{K}")
    all_keys = np.concatenate([surv_keys, win_keys])
    c, e, cl = oracle.count_keys(rs.bases, rs.quals, rs.offsets, p, all_keys, threads=threads)
    # survivors: exact values
    assert (c[:3000] == cnt[pick]).all()
    assert (e[:3000] == ext[pick]).all()
    assert (cl[:3000] == res.cls[pick]).all()
    # window k-mers: present iff count >= min_count, with the same values
    packed = encode(win_keys)
    pos = np.searchsorted(sk, packed)
    pos = np.minimum(pos, n - 1)
    found = sk[pos] == packed
    want_present = c[3000:] >= p.min_count
    assert (found == want_present).all()
    idx = order[pos[found]]
    assert (cnt[idx] == c[3000:][found]).all()
    assert (ext[idx] == e[3000:][found]).all()
    assert (res.cls[idx] == cl[3000:][found]).all()
