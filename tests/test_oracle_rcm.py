"""Pins of the RCM oracle (Section 2, Example 2; Section 3) and of the
symmetric permutation P A P^T."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import dacsr as D
from oracle import rcm as R


def _graph_csr(n, edges):
    rows, cols = [], []
    for a, b in edges:
        rows += [a, b]
        cols += [b, a]
    rows += list(range(n))
    cols += list(range(n))
    return W.from_coo(n, rows, cols)


def _hand_examples():
    import os
    from conftest import GOLDEN
    out = []
    with open(os.path.join(GOLDEN, "rcm_hand_examples.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, n, edges, perm = [p.strip() for p in line.split("|")]
                e = [tuple(int(t) for t in s.split("-")) for s in edges.split()]
                out.append((name, int(n), e, [int(t) for t in perm.split()]))
    return out


@pytest.mark.parametrize("name,n,edges,perm", _hand_examples())
def test_hand_worked(name, n, edges, perm):
    rp, c, _ = _graph_csr(n, edges)
    assert R.rcm_order(n, rp, c).tolist() == perm


def _perm_bandwidth(n, rp, c, perm):
    rp2, c2, _ = R.permute_symmetric(n, rp, c, np.ones(len(c)), perm)
    return D.bandwidth(n, rp2, c2)


def test_path_and_cycle_scrambled():
    rng = np.random.default_rng(1)
    n = 60
    lab = rng.permutation(n)
    path = [(lab[i], lab[i + 1]) for i in range(n - 1)]
    rp, c, _ = _graph_csr(n, path)
    assert D.bandwidth(n, rp, c) > 1
    assert _perm_bandwidth(n, rp, c, R.rcm_order(n, rp, c)) == 1
    cyc = path + [(lab[-1], lab[0])]
    rp, c, _ = _graph_csr(n, cyc)
    assert _perm_bandwidth(n, rp, c, R.rcm_order(n, rp, c)) == 2


def test_grid_level_bound():
    k = 9
    rng = np.random.default_rng(2)
    lab = rng.permutation(k * k)
    edges = []
    for i in range(k):
        for j in range(k):
            if i + 1 < k:
                edges.append((lab[i * k + j], lab[(i + 1) * k + j]))
            if j + 1 < k:
                edges.append((lab[i * k + j], lab[i * k + j + 1]))
    rp, c, _ = _graph_csr(k * k, edges)
    w = _perm_bandwidth(k * k, rp, c, R.rcm_order(k * k, rp, c))
    # optimal bandwidth of the k x k grid is k; a corner start gives
    # anti-diagonal levels of width <= k, hence w <= 2k - 1
    assert k <= w <= 2 * k - 1


def _level_bound(n, rp, c, perm):
    """max over consecutive BFS levels (|L_i| + |L_i+1|) - 1 for the level
    structure rooted at each component's first vertex in CM order."""
    ptr, adj, deg = R.symmetric_graph(n, rp, c)
    cm = list(perm[::-1])
    seen = set()
    bound = 0
    for v in cm:
        if v in seen:
            continue
        levels = R.level_structure(int(v), ptr, adj)
        for L in levels:
            seen.update(L)
        for a, b in zip(levels, levels[1:]):
            bound = max(bound, len(a) + len(b) - 1)
    return bound


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_small(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 8))
    m = int(rng.integers(1, n * (n - 1) // 2 + 1))
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    sel = rng.choice(len(pairs), size=m, replace=False)
    edges = [pairs[i] for i in sel]
    rp, c, _ = _graph_csr(n, edges)
    perm = R.rcm_order(n, rp, c)
    assert sorted(perm.tolist()) == list(range(n))
    w = _perm_bandwidth(n, rp, c, perm)
    w_opt = min(_perm_bandwidth(n, rp, c, np.array(p)) for p in itertools.permutations(range(n)))
    assert w_opt <= w <= max(_level_bound(n, rp, c, perm), w_opt)


@pytest.mark.parametrize("seed", range(4))
def test_permute_symmetric_dense(seed):
    rng = np.random.default_rng(seed)
    n = 17
    nnz = 60
    rows, cols = rng.integers(0, n, nnz), rng.integers(0, n, nnz)
    vals = rng.standard_normal(nnz)
    rp, c, v = W.from_coo(n, rows, cols, vals)
    # deduplicate for the dense comparison
    A = np.zeros((n, n))
    for r in range(n):
        for i in range(rp[r], rp[r + 1]):
            A[r, c[i]] += v[i]
    perm = rng.permutation(n)
    rp2, c2, v2 = R.permute_symmetric(n, rp, c, v, perm)
    B = np.zeros((n, n))
    for r in range(n):
        assert np.all(np.diff(c2[rp2[r]:rp2[r + 1]]) >= 0)
        for i in range(rp2[r], rp2[r + 1]):
            B[r, c2[i]] += v2[i]
    assert np.array_equal(B, A[np.ix_(perm, perm)])


def test_scrambled_laplacian_restored():
    m = 14
    rng = W.rng_for(2, 1)
    rp, c, v = W.laplace3d_7pt(m, scrambled=True, rng=rng)
    n = m ** 3
    assert D.bandwidth(n, rp, c) > n // 2
    perm = R.rcm_order(n, rp, c)
    w = _perm_bandwidth(n, rp, c, perm)
    # at most a few grid planes: the natural order has w = m^2
    assert w <= 2 * m * m
    # cross-check against SciPy's RCM (a different implementation; loose)
    sp = pytest.importorskip("scipy.sparse")
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    A = sp.csr_matrix((v, c, rp), shape=(n, n))
    p2 = reverse_cuthill_mckee(A, symmetric_mode=True)
    w2 = _perm_bandwidth(n, rp, c, p2)
    assert w <= 1.5 * w2 + 2


def _selfloop_case():
    """Path 0-1-2-3 with a self loop on vertex 0 only, worked by hand.  Self
    loops are not edges: degrees 1, 2, 2, 1; the minimum (degree, index) is
    0; L(0) = [0][1][2][3] and the last level's vertex 3 has no larger
    eccentricity, so CM runs 0, 1, 2, 3 and the reversal gives 3, 2, 1, 0.
    Counting the loop would give vertex 0 degree 2, start at 3 and return
    0, 1, 2, 3."""
    rp, c, _ = W.from_coo(4, [0, 0, 1, 1, 2, 2, 3], [0, 1, 0, 2, 1, 3, 2])
    return "selfloop", 4, rp, c, [3, 2, 1, 0]


def _pinned_cases():
    out = []
    for name, n, edges, perm in _hand_examples():
        rp, c, _ = _graph_csr(n, edges)
        out.append((name, n, rp, c, perm))
    out.append(_selfloop_case())
    return out


def test_selfloop_hand_example():
    name, n, rp, c, perm = _selfloop_case()
    assert R.rcm_order(n, rp, c).tolist() == perm


def _cm_sorted_by(key):
    def cm(start, ptr, adj, deg, visited):
        order = [start]
        visited[start] = True
        queue = [start]
        while queue:
            v = queue.pop(0)
            nbrs = [u for u in adj[ptr[v]:ptr[v + 1]].tolist() if not visited[u]]
            nbrs.sort(key=lambda t: key(int(deg[t]), t))
            for u in nbrs:
                visited[u] = True
                order.append(u)
                queue.append(u)
        return order
    return cm


def _george_liu(pick, moves_on_equal=False):
    def pp(start, ptr, adj, deg):
        v = start
        levels = R.level_structure(v, ptr, adj)
        for _ in range(4 * len(ptr)):
            u = pick(levels[-1], deg)
            lu = R.level_structure(u, ptr, adj)
            if len(lu) > len(levels) or (moves_on_equal and len(lu) == len(levels) and u != v):
                v, levels = u, lu
            else:
                break
        return v
    return pp


def _graph_with_loops_in_degree(n, rowptr, col):
    ptr, adj, deg = ORIG_SYMMETRIC_GRAPH(n, rowptr, col)
    r = D.entry_rows(n, rowptr)
    has_loop = np.zeros(n, dtype=np.int64)
    has_loop[r[r == np.asarray(col)]] = 1
    return ptr, adj, deg + has_loop


ORIG_SYMMETRIC_GRAPH = R.symmetric_graph


@pytest.mark.parametrize("mistake", ["not_reversed", "ties_index_descending", "degree_descending",
                                     "neighbours_by_index", "no_george_liu",
                                     "george_liu_moves_on_equal", "last_level_by_index",
                                     "self_loops_in_degree"])
def test_planted_mistakes_are_caught(mistake, monkeypatch):
    """Each plausible slip in the ordering changes at least one hand-worked
    permutation (the mistake is planted in the oracle, on the CPU)."""
    order = R.rcm_order
    if mistake == "not_reversed":
        order = lambda n, rp, c: R.rcm_order(n, rp, c)[::-1]
    elif mistake == "ties_index_descending":
        monkeypatch.setattr(R, "cuthill_mckee_from", _cm_sorted_by(lambda d, t: (d, -t)))
    elif mistake == "degree_descending":
        monkeypatch.setattr(R, "cuthill_mckee_from", _cm_sorted_by(lambda d, t: (-d, t)))
    elif mistake == "neighbours_by_index":
        monkeypatch.setattr(R, "cuthill_mckee_from", _cm_sorted_by(lambda d, t: t))
    elif mistake == "no_george_liu":
        monkeypatch.setattr(R, "pseudo_peripheral", lambda start, ptr, adj, deg: start)
    elif mistake == "george_liu_moves_on_equal":
        monkeypatch.setattr(R, "pseudo_peripheral",
                            _george_liu(lambda last, deg: min(last, key=lambda t: (int(deg[t]), t)),
                                        moves_on_equal=True))
    elif mistake == "last_level_by_index":
        monkeypatch.setattr(R, "pseudo_peripheral", _george_liu(lambda last, deg: min(last)))
    else:
        monkeypatch.setattr(R, "symmetric_graph", _graph_with_loops_in_degree)
    wrong = [name for name, n, rp, c, perm in _pinned_cases()
             if np.asarray(order(n, rp, c)).tolist() != perm]
    assert wrong, mistake


def test_inverse_permutation():
    """iperm[perm[i]] = i, by hand and on random permutations (both ways)."""
    assert R.inverse_permutation([2, 0, 1]).tolist() == [1, 2, 0]
    assert R.inverse_permutation([0]).tolist() == [0]
    rng = np.random.default_rng(7)
    for n in (1, 2, 17, 1000):
        perm = rng.permutation(n)
        ip = R.inverse_permutation(perm)
        assert np.array_equal(ip[perm], np.arange(n))
        assert np.array_equal(perm[ip], np.arange(n))
