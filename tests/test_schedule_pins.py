"""Pins for two closed forms the CUDA schedules rely on, checked on the
oracle's own trees and on exact arithmetic (no GPU).

1. Record offsets without a scan.  A node's record takes 3 + (its internal
   children) four-word units (12 / 16 / 20 words).  The segment schedule
   writes the offset of the node at id a of body j as 4a - j - delta,
   delta = 1 when leaf g = a - (off[j] - j) is the right child of split
   g - 1 (leaf i hangs from split i - 1 or split i of the bisection tree,
   Sec. 2.1).  The test sums the sizes over every node of many trees and
   compares at every id.

2. Tree keys from one fused multiply-add.  The per-body tree kernels take
   floor(p s + c) (s = 2^21 / (hi - lo), c = -lo s, one FP64 fused
   multiply-add) unless the value lies within 2^-beta of an integer, where
   B = 2^-27 + |lo| s 2^-51 < 2^-beta bounds its distance from 2^21 times
   the exact FP64 quotient; such beads, and those in the top cell, take
   the exact formula (Sec. 2.1 quantisation, as the oracle computes it).
   The decision is restated here with the fused multiply-add evaluated
   exactly (rationals, rounded once), on beads on and one ulp beside cell
   boundaries and bodies up to 1e12 times their size from the origin; its
   floor must equal the exact formula's everywhere.
"""
import math
import struct
from fractions import Fraction

import numpy as np

import oracle
from paper_1708_08427_gb300 import workloads as W

QBITS = 21


# ------------------------------------------------------------ 1. offsets
def _bodies():
    rng = np.random.default_rng(11)
    g = np.arange(64)
    pts = [
        rng.uniform(-1, 1, (3, 3)),
        np.c_[np.arange(40) * 0.25, np.arange(40) * 0.5, np.full(40, 1.0)],
        np.c_[g % 4, (g // 4) % 4, g // 16].astype(float),
        rng.uniform(0, 1, (700, 3)),
    ]
    bt = W.shell_batch(m=25, nmin=3, nmax=2500, seed=8)
    pts += [np.stack(bt.body(j), 1) for j in range(bt.m)]
    return pts


def test_record_offsets_closed_form():
    off, run, j_all = 0, 0, 0
    checked = 0
    for j, P in enumerate(_bodies()):
        n = P.shape[0]
        t = oracle.Body(P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy()).tree()
        left, right = t["left"], t["right"]
        nb = off - j
        for g in range(n - 1):
            a = nb + g
            delta = int(g > 0 and right[g - 1] < 0 and -1 - right[g - 1] == g)
            assert run == 4 * a - j - delta, (j, g)
            run += 3 + int(left[g] >= 0) + int(right[g] >= 0)
            checked += 1
        off += n
        j_all = j + 1
    assert run == 4 * off - 5 * j_all  # the total, written after the last offset
    assert checked > 5000


# ------------------------------------------------------------ 2. the keys
def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _exact(p, lo, hi):
    t = (p - lo) / (hi - lo)
    return min(math.floor(t * 2.0 ** QBITS), 2 ** QBITS - 1)


def _axis(lo, hi):
    s = 2.0 ** QBITS / (hi - lo)
    c = -lo * s
    B = 2.0 ** -27 + abs(lo) * s * 2.0 ** -51
    beta = -math.frexp(B)[1]  # B < 2^-beta (frexp: B = m 2^e, m in [1/2, 1))
    return s, c, max(beta, 0)


def _fma_key(p, lo, hi, ax, used):
    s, c, beta = ax
    v = float(Fraction(p) * Fraction(s) + Fraction(c))  # one rounding
    b = _bits(v)
    e = ((b >> 52) & 0x7FF) - 1023
    if (b >> 63) == 0 and beta > 0:
        M = (b & ((1 << 52) - 1)) | (1 << 52)
        if 0 <= e <= 20:
            fb = 52 - e
            ip, fr = M >> fb, M & ((1 << fb) - 1)
            margin = 1 << (fb - beta) if fb > beta else 1
            if margin < fr < (1 << fb) - margin and ip < 2 ** QBITS - 1:
                used[0] += 1
                return ip
        elif -beta <= e < 0:
            if e <= -2 or (1 << 53) - M >= (1 << (53 - beta)):
                used[0] += 1
                return 0
    used[1] += 1
    return _exact(p, lo, hi)


def test_fma_keys_equal_exact_formula():
    rng = np.random.default_rng(5)
    used = [0, 0]
    n = 0
    for trial in range(1500):
        off = [0.0, 1.0, -3.7, 1e3, -1e5, 1e6, 1e9, 1e12, 1e-3][trial % 9]
        size = [1.0, 1e-3, 1e-6, 37.0, 1e4][trial % 5]
        lo = off + rng.uniform(-1, 1) * size
        hi = lo + size * rng.uniform(0.5, 2)
        if not hi > lo:
            continue
        ax = _axis(lo, hi)
        w = (hi - lo) / 2.0 ** QBITS
        for k in range(12):
            if k < 3:
                p = rng.uniform(lo, hi)
            else:
                base = lo + int(rng.integers(0, 2 ** QBITS)) * w
                p = [base, math.nextafter(base, math.inf), math.nextafter(base, -math.inf)][k % 3]
            p = min(max(p, lo), hi)
            assert _fma_key(p, lo, hi, ax, used) == _exact(p, lo, hi), (p, lo, hi)
            n += 1
        for p in (lo, hi):  # the corners: the exact formula's clamp
            assert _fma_key(p, lo, hi, ax, used) == _exact(p, lo, hi)
    # both paths were exercised
    assert used[0] > 1000 and used[1] > 1000, used


def test_fma_keys_take_the_fast_path_on_generic_beads():
    rng = np.random.default_rng(6)
    used = [0, 0]
    for _ in range(300):
        lo = rng.uniform(-50, 50)
        hi = lo + rng.uniform(1, 40)
        ax = _axis(lo, hi)
        for p in rng.uniform(lo, hi, 20):
            assert _fma_key(float(p), lo, hi, ax, used) == _exact(float(p), lo, hi)
    assert used[1] == 0, used  # no uniform bead within 2^-26 of a boundary here
