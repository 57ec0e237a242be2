"""RCM ordering and P A P^T through the C ABI against the oracle
(Section 2, Example 2; Section 3): the host ordering bit for bit, the device
permutation bit for bit (pattern and values of every dtype), and the
bandwidths against Eq. (2)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import dacsr as OD
from oracle import rcm as OR

from test_oracle_rcm import _graph_csr, _hand_examples

pytestmark = pytest.mark.gpu


def _scrambled(n, rp, col, val, rng):
    lab = rng.permutation(n).astype(np.int32)          # old vertex v -> label lab[v]
    perm = np.argsort(lab).astype(np.int32)            # new -> old
    return OR.permute_symmetric(n, rp, col, val, perm)


def _order_cases():
    rng = np.random.default_rng(3)
    out = []
    for name, n, edges, _ in _hand_examples():
        rp, c, _ = _graph_csr(n, edges)
        out.append((name, n, rp, c))
    rp, c, v = W.laplace2d_5pt(30)
    out.append(("lap2d_30_scrambled", 900) + _scrambled(900, rp, c, v, rng)[:2])
    n = 3000
    rp, c, v = W.random_banded(n, 200, rng)
    out.append(("banded_3000_scrambled", n) + _scrambled(n, rp, c, v, rng)[:2])
    # nonsymmetric pattern, several components, isolated vertices, empty rows
    rows = [0, 0, 1, 5, 5, 7, 9, 9, 12]
    cols = [3, 0, 4, 2, 8, 7, 11, 1, 12]
    rp, c, _ = W.from_coo(14, rows, cols)
    out.append(("nonsym_components", 14, rp, c))
    rp, c, v = W.laplace3d_7pt(16, scrambled=True, rng=np.random.default_rng(9))
    out.append(("lap3d_16_scrambled", 16 ** 3, rp, c))
    return out


@pytest.mark.parametrize("case", _order_cases(), ids=lambda c: c[0])
def test_rcm_order_bit_exact(D, case):
    name, n, rp, c = case
    perm, wb, wa = D.damn_rcm_order(rp, c)
    ref = OR.rcm_order(n, rp, c)
    assert np.array_equal(perm, ref)
    assert wb == OD.bandwidth(n, rp, c)
    rp2, c2, _ = OR.permute_symmetric(n, rp, c, np.zeros(len(c)), ref)
    assert wa == OD.bandwidth(n, rp2, c2)


def test_rcm_order_rejects_bad_pattern(D):
    rp = np.array([0, 1, 2], dtype=np.int32)
    with pytest.raises(D.DamnError):
        D.damn_rcm_order(rp, np.array([0, 5], dtype=np.int32))      # column out of range
    with pytest.raises(D.DamnError):
        D.damn_rcm_order(np.array([0, 2, 1], dtype=np.int32), np.array([0, 1], dtype=np.int32))


def _perm_matrix(rng, n):
    """Rows of length 0..1500 (empty, <32, >32, >1024) with repeated columns."""
    lens = rng.integers(0, 40, size=n)
    lens[rng.choice(n, 5, replace=False)] = 0
    lens[rng.choice(n, 4, replace=False)] = [33, 64, 700, 1500]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    col = rng.integers(0, n, size=int(rp[-1])).astype(np.int32)
    dup = rng.random(col.size) < 0.1
    col[1:][dup[1:]] = col[:-1][dup[1:]]                # repeated columns in a row
    val = rng.standard_normal(col.size)
    return rp.astype(np.int32), col, val


@pytest.mark.parametrize("dt", [torch.float64, torch.float32, torch.bfloat16, None])
def test_permute_sym_bit_exact(D, cuda_dev, dt):
    rng = np.random.default_rng(11)
    n = 5000
    rp, col, val = _perm_matrix(rng, n)
    perm = rng.permutation(n).astype(np.int32)
    tv = None if dt is None else torch.from_numpy(val).to(cuda_dev).to(dt)
    rp_o, col_o, val_o = D.damn_permute_sym(torch.from_numpy(rp).to(cuda_dev),
                                            torch.from_numpy(col).to(cuda_dev), tv,
                                            torch.from_numpy(perm).to(cuda_dev))
    torch.cuda.synchronize()
    vref = np.arange(col.size)                          # permute positions, then values
    rp_r, col_r, pos_r = OR.permute_symmetric(n, rp, col, vref, perm)
    assert np.array_equal(rp_o.cpu().numpy(), rp_r)
    assert np.array_equal(col_o.cpu().numpy(), col_r)
    if dt is not None:
        assert torch.equal(val_o.cpu(), tv.cpu()[torch.from_numpy(pos_r)])
    assert D.damn_device_status(reset=True) == D.DAMN_OK


def test_permute_sym_invalid_perm_reports(D, cuda_dev):
    n = 100
    rp, c, v = W.laplace2d_5pt(10)
    perm = np.arange(n, dtype=np.int32)
    perm[7] = perm[3]                                    # repeated value: not a permutation
    D.damn_device_status(reset=True)
    D.damn_permute_sym(torch.from_numpy(rp).to(cuda_dev), torch.from_numpy(c).to(cuda_dev),
                       torch.from_numpy(v).to(cuda_dev), torch.from_numpy(perm).to(cuda_dev))
    assert D.damn_device_status(reset=True) == D.DAMN_ERR_INVALID_ARG
    perm = np.arange(n, dtype=np.int32)
    perm[0] = n + 3                                      # out of range
    D.damn_permute_sym(torch.from_numpy(rp).to(cuda_dev), torch.from_numpy(c).to(cuda_dev),
                       None, torch.from_numpy(perm).to(cuda_dev))
    assert D.damn_device_status(reset=True) == D.DAMN_ERR_INVALID_ARG


def test_permute_sym_empty(D, cuda_dev):
    rp = torch.zeros(1, dtype=torch.int32, device=cuda_dev)
    e = torch.zeros(0, dtype=torch.int32, device=cuda_dev)
    rp_o, col_o, _ = D.damn_permute_sym(rp, e, None, e)
    torch.cuda.synchronize()
    assert rp_o.cpu().tolist() == [0] and col_o.numel() == 0


def test_rcm_permute_restores_fit_medium(D, cuda_dev):
    """Scrambled 40^3 7-point Laplacian: bandwidth far beyond 2^15, RCM
    brings it back into int16 range; ordering and B equal the oracle's."""
    m = 40
    n = m ** 3
    rp, c, v = W.laplace3d_7pt(m, scrambled=True, rng=np.random.default_rng(4))
    assert OD.bandwidth(n, rp, c) > 32767
    t = lambda a: torch.from_numpy(a).to(cuda_dev)
    perm, rp_o, col_o, val_o, info = D.damn_rcm_permute(t(rp), t(c), t(v))
    ref = OR.rcm_order(n, rp, c)
    assert np.array_equal(perm.cpu().numpy(), ref)
    rp_r, c_r, v_r = OR.permute_symmetric(n, rp, c, v, ref)
    assert np.array_equal(rp_o.cpu().numpy(), rp_r)
    assert np.array_equal(col_o.cpu().numpy(), c_r)
    assert np.array_equal(val_o.cpu().numpy(), v_r)
    assert info["w_before"] == OD.bandwidth(n, rp, c)
    assert info["w_after"] == OD.bandwidth(n, rp_r, c_r) <= 32767
    assert OD.fit_check(n, n, rp_r, c_r).fits


def test_rcm_permute_full_size_scrambled_128(D, cuda_dev):
    """128^3 scrambled 7-point Laplacian (2,097,152 rows): perm is a
    permutation, B equals the oracle's P A P^T for that perm, the reported
    bandwidths match Eq. (2), and B fits DA-CSR-16."""
    m = 128
    n = m ** 3
    rp, c, v = W.laplace3d_7pt(m, scrambled=True, rng=W.rng_for(2, 1))
    t = lambda a: torch.from_numpy(a).to(cuda_dev)
    perm, rp_o, col_o, val_o, info = D.damn_rcm_permute(t(rp), t(c), t(v))
    p = perm.cpu().numpy()
    assert np.array_equal(np.sort(p), np.arange(n))
    rp_r, c_r, v_r = OR.permute_symmetric(n, rp, c, v, p)
    assert np.array_equal(rp_o.cpu().numpy(), rp_r)
    assert np.array_equal(col_o.cpu().numpy(), c_r)
    assert np.array_equal(val_o.cpu().numpy(), v_r)
    assert info["w_before"] == OD.bandwidth(n, rp, c)
    assert info["w_after"] == OD.bandwidth(n, rp_r, c_r)
    assert info["w_after"] <= 32767
