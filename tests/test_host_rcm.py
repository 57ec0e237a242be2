"""The library's host-side RCM ordering (damn_rcm_order: host arrays in and
out, no device work) against the oracle, on the CPU: the permutation bit for
bit under the fixed reading of Section 2, Example 2 and Section 3 (graph of
A + A^T, components by smallest vertex, George-Liu start, neighbours by
(degree, index), reversed), and the bandwidths of Eq. (2) before and after."""
import numpy as np
import pytest

import workloads as W
from oracle import dacsr as OD
from oracle import rcm as OR

from test_gpu_rcm import _order_cases


@pytest.fixture(scope="module")
def D():
    from paper_2307_06305_gb300 import build as B
    B.build()
    from paper_2307_06305_gb300 import damn
    return damn


def _extra_cases():
    out = []
    rp, c, _ = W.laplace3d_7pt(32, scrambled=True, rng=np.random.default_rng(32))
    out.append(("lap3d_32_scrambled", 32 ** 3, rp, c))
    rng = np.random.default_rng(5)
    n = 20000
    rp, c, _ = W.random_banded(n, 50, rng)
    lab = rng.permutation(n).astype(np.int32)
    rp, c, _ = OR.permute_symmetric(n, rp, c, np.zeros(len(c)), np.argsort(lab).astype(np.int32))
    out.append(("banded_20000_scrambled", n, rp, c))
    # a single vertex, and vertices without any edge
    out.append(("one_vertex", 1, np.array([0, 0], dtype=np.int32), np.zeros(0, dtype=np.int32)))
    out.append(("edgeless", 6, np.zeros(7, dtype=np.int32), np.zeros(0, dtype=np.int32)))
    # self loops only (dropped from the graph)
    out.append(("self_loops", 4, np.arange(5, dtype=np.int32), np.arange(4, dtype=np.int32)))
    return out


@pytest.mark.parametrize("case", _order_cases() + _extra_cases(), ids=lambda c: c[0])
def test_host_rcm_order_bit_exact(D, case):
    name, n, rp, c = case
    perm, wb, wa = D.damn_rcm_order(rp, c)
    ref = OR.rcm_order(n, rp, c)
    assert np.array_equal(perm, ref)
    assert sorted(perm.tolist()) == list(range(n))
    assert wb == OD.bandwidth(n, rp, c)
    rp2, c2, _ = OR.permute_symmetric(n, rp, c, np.zeros(len(c)), ref)
    assert wa == OD.bandwidth(n, rp2, c2)


def test_host_rcm_restores_int16_fit(D):
    """A scrambled 40^3 grid (half-bandwidth about n) is brought back well
    inside int16 range by the ordering."""
    m = 40
    rp, c, _ = W.laplace3d_7pt(m, scrambled=True, rng=np.random.default_rng(40))
    perm, wb, wa = D.damn_rcm_order(rp, c)
    assert wb > 32767 and wa < 2 * m * m


def test_host_rcm_rejects_bad_pattern(D):
    rp = np.array([0, 1, 2], dtype=np.int32)
    with pytest.raises(D.DamnError):
        D.damn_rcm_order(rp, np.array([0, 5], dtype=np.int32))      # column out of range
    with pytest.raises(D.DamnError):
        D.damn_rcm_order(np.array([0, 2, 1], dtype=np.int32), np.array([0, 1], dtype=np.int32))
