"""Host side of the maximum-determinant completion (Section 7.1.1): sizes of
the dense per-component output and of the device scratch.  No GPU call."""
import numpy as np

from paper_1707_05058_gb300 import workloads as W


def test_completion_sizes_single_component(lib):
    prob = W.workload(0)
    P = lib.Problem(prob)
    sb, we, offs = P.completion_sizes()
    assert int(P.info["ncomp"]) == 1
    assert we == prob.n ** 2 and list(offs) == [0, prob.n ** 2]
    assert sb > 0 and sb % 256 == 0


def test_completion_sizes_direct_sum(lib):
    parts = [W.banded(50, 3, 10, seed=1), W.workload(0), W.maxcut_cycle(7)]
    prob = W.direct_sum(parts)
    P = lib.Problem(prob)
    sb, we, offs = P.completion_sizes()
    vc, _ = P.components()
    sizes = np.bincount(vc, minlength=int(P.info["ncomp"]))
    assert list(sizes) == [p.n for p in parts]
    np.testing.assert_array_equal(offs, np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)]))
    assert we == offs[-1]
