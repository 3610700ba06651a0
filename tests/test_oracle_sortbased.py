"""The oracle against a second CPU implementation of the same definition,
written another way: every window of every read laid out as a row of base
codes (numpy), canonicalised row by row, then sorted and run-length grouped
(np.unique) instead of inserted into an ordered map; tallies accumulated by
scatter-add; sides classified by a vectorised form of the rule of Sec. II-C.

On the single-genome reads (20 000 x 150 bp from a 100 kbp genome) at k = 21
and the multi-k ladder k = 21, 33, 55, 77, 99 on the same reads, the two must
agree on every survivor (key, count, the eight tallies, both classes) and on
the window and distinct totals.  The two share no code: this file does not
use the oracle's parsing, reverse complement, map or classifier.
"""
import numpy as np
import pytest

import oracle
import synth

CODE = np.full(256, 4, dtype=np.uint8)  # 4 = not a base
for i, b in enumerate(b"ACGT"):
    CODE[b] = i
LETTER = np.frombuffer(b"ACGT", np.uint8)


def sort_based(bases, quals, offsets, k, min_count=2, qual_offset=33, qual_threshold=20, t_base=2, num=1, den=10):
    codes = CODE[bases]
    offs = offsets.astype(np.int64)
    lens = np.diff(offs)
    nwin = np.maximum(lens - k + 1, 0)
    read = np.repeat(np.arange(len(lens)), nwin)
    first = np.repeat(offs[:-1], nwin)
    start = first + (np.arange(int(nwin.sum())) - np.repeat(np.cumsum(nwin) - nwin, nwin))
    rows = codes[start[:, None] + np.arange(k)[None, :]]  # (windows, k)
    ok = (rows < 4).all(axis=1)
    rows, start, read = rows[ok], start[ok], read[ok]
    end = offs[1:][read]
    rc = 3 - rows[:, ::-1]
    differ = rows != rc
    pos = differ.argmax(axis=1)
    idx = np.arange(len(rows))
    flip = differ.any(axis=1) & (rc[idx, pos] < rows[idx, pos])
    canon = np.where(flip[:, None], rc, rows)
    # extension bases on the read: before and after the window, if present, a base and of high quality
    hq = lambda p: (quals[p].astype(np.int64) - qual_offset) >= qual_threshold
    has_l = start > offs[:-1][read]
    lp = np.where(has_l, start - 1, 0)
    lb = codes[lp]
    l_ok = has_l & (lb < 4) & hq(lp)
    has_r = start + k < end
    rp = np.where(has_r, start + k, 0)
    rb = codes[rp]
    r_ok = has_r & (rb < 4) & hq(rp)
    # on a flipped window the sides swap and the bases are complemented
    left_b = np.where(flip, 3 - rb, lb)
    left_ok = np.where(flip, r_ok, l_ok)
    right_b = np.where(flip, 3 - lb, rb)
    right_ok = np.where(flip, l_ok, r_ok)
    keys = LETTER[canon].reshape(len(canon) * k).view(f"S{k}") if len(canon) else np.empty(0, f"S{k}")
    uniq, inv, count = np.unique(keys, return_inverse=True, return_counts=True)
    ext = np.zeros((len(uniq), 8), dtype=np.int64)
    np.add.at(ext, (inv[left_ok], left_b[left_ok].astype(np.int64)), 1)
    np.add.at(ext, (inv[right_ok], 4 + right_b[right_ok].astype(np.int64)), 1)
    keep = count >= min_count
    uniq, count, ext = uniq[keep], count[keep], ext[keep]
    cls = np.zeros((len(uniq), 2), dtype=np.uint8)
    for side in range(2):
        n = ext[:, 4 * side:4 * side + 4]
        m = n.argmax(axis=1)
        top = n.max(axis=1)
        ties = (n == top[:, None]).sum(axis=1)
        alt = n.sum(axis=1) - top
        unique = alt * den <= np.maximum(t_base * den, num * count)
        c = np.where(top == 0, 5, np.where(ties > 1, 4, np.where(unique, m, 4)))
        cls[:, side] = c
    return uniq, count, ext, cls, int(ok.sum()), int(len(keep))


@pytest.fixture(scope="module")
def reads():
    return synth.generate(synth.SINGLE_GENOME)


@pytest.mark.parametrize("k", [21, 33, 55, 77, 99])
def test_oracle_equals_a_sort_based_count(reads, k):
    keys, count, ext, cls, windows, distinct = sort_based(reads.bases, reads.quals, reads.offsets, k)
    got = oracle.run(reads.bases, reads.quals, reads.offsets, oracle.Params(k=k))
    assert got.windows == windows and got.distinct == distinct
    assert len(got.keys) == len(keys) > 1000
    assert (got.keys == keys).all()
    assert (got.count.astype(np.int64) == count).all()
    assert (got.ext.astype(np.int64) == ext).all()
    assert (got.cls == cls).all()
