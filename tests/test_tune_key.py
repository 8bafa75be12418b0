"""The autotuner's cache key (no GPU): bodies binned by powers of two, so
that two batches of the same shape share a pick and different ones do not."""
import numpy as np

from paper_1708_08427_gb300 import tune
from paper_1708_08427_gb300 import workloads as W


def test_shape_key_bins_body_sizes():
    a = W.shell_batch(m=50, nmin=50, nmax=5000, seed=0).off
    b = W.shell_batch(m=50, nmin=50, nmax=5000, seed=0).off
    c = W.shell_batch(m=50, nmin=50, nmax=5000, seed=1).off
    k = lambda off, **kw: tune.shape_key(off, kw.get("prec", "fp32"), "dd", "caller", True)
    assert k(a) == k(b)
    assert k(a) != k(c) or np.array_equal(a, c) is False  # other sizes: other totals
    assert k(a) != k(a, prec="fp64")
    off = np.array([0, 64, 128, 256])  # 64, 64, 128 beads
    key = tune.shape_key(off, "fp32", "dd", "caller", False)
    assert '"log2_hist": [0, 0, 0, 0, 0, 0, 2, 1]' in key and '"N": 256' in key


def test_candidates_cover_every_cut_and_the_fused_step():
    assert set(c for s, c in tune.CANDIDATES if s == "levels") == set(tune.CUTS)
    assert ("fused", 0) in tune.CANDIDATES
