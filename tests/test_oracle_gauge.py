"""Pins of the oracle's tree-gauge compression (projector form) against independent truths.

  * r = 0: the projector form inserts exactly the plain compression
    (A P_L = Q_A U_k s_k^1/2), so it reproduces oracle.approx to rounding;
  * a loop-free network with its whole environment in the gauge: each side
    of a cut bond reduces to a vector, so the core R_A L_B has rank one and
    a compression to chi = 1 loses nothing (exact Z), while r = 0 does lose;
  * the paper's accuracy claim: on the 8x8 Ising model at chi = 4 the error
    against the row transfer matrix falls as r grows;
  * Algorithm 2: the spanning tree stays within distance r and within the
    allowed nodes, reaches every such node once, closest first;
planted mistakes (absorbing R factors outwards, no s^-1/2 in the projectors)
must break a pin.
"""
import numpy as np
import pytest

from oracle import approx, exact, gauge
from tn_inputs import networks as nw
from tn_inputs import trees as tr


@pytest.mark.parametrize("chi", [4, 16])
def test_r0_projector_form_equals_plain_compression_ising(chi):
    n, e = nw.square_lattice(8, 8)
    net = nw.ising_network(n, e, 0.44)
    tree = tr.boundary_rows(8, 8)
    a = approx.contract(net, tree, chi)
    g = gauge.contract_gauged(net, tree, chi, 0)
    assert g.compressions == a.compressions and abs(g.logabs - a.logabs) < 1e-12 * abs(a.logabs)


def test_r0_projector_form_equals_plain_compression_positive_random():
    n, e = nw.square_lattice(6, 7)
    net = nw.random_network(n, e, 3, seed=4, dist="uniform", lam=0.0)
    tree = tr.boundary_rows(6, 7)
    a = approx.contract(net, tree, 5)
    g = gauge.contract_gauged(net, tree, 5, 0)
    assert abs(g.logabs - a.logabs) < 1e-12 * abs(a.logabs)


def tree_case(seed):
    n, e = nw.random_tree_graph(12, seed=seed)
    net = nw.random_network(n, e, 3, seed=seed + 5, dist="uniform", lam=0.1)
    return net, tr.from_pairs(net.bonds, tr.sequential_pairs(n), "early")


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_full_tree_gauge_on_a_loop_free_network_is_exact_at_chi_1(seed):
    net, t = tree_case(seed)
    z = approx.contract_exact(net, t)
    g = gauge.contract_gauged(net, t, 1, 1000, include_inputs=True)
    assert g.compressions > 0
    assert g.sign == z.sign and abs(g.logabs - z.logabs) < 1e-12 * max(1.0, abs(z.logabs))
    plain = gauge.contract_gauged(net, t, 1, 0, include_inputs=True)
    assert abs(plain.logabs - z.logabs) > 1e-6


def test_error_falls_with_gauge_distance_ising_8x8():
    n, e = nw.square_lattice(8, 8)
    net = nw.ising_network(n, e, 0.44)
    tree = tr.boundary_rows(8, 8)
    tm = exact.ising_transfer_2d(8, 8, 0.44)["lnZ"]
    errs = [abs(gauge.contract_gauged(net, tree, 4, r).logabs - tm) for r in (0, 1, 2, 4)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3 * errs[0]


def test_spanning_tree_algorithm_2():
    # a 5 x 5 grid graph of "tensors" with bond size 2
    n, e = nw.square_lattice(5, 5)
    net = nw.random_network(n, e, 2, seed=0)
    bonds = {t: list(b) for t, b in enumerate(net.bonds)}
    dims = {b: 2 for b in range(len(net.bond_dims))}
    # breadth-first distances from {12, 13} in the graph without the excluded node 7
    adj = {v: [w for w in range(n) if w != v and set(bonds[v]) & set(bonds[w])] for v in range(n)}
    dist = {12: 0, 13: 0}
    frontier = [12, 13]
    while frontier:
        nxt = []
        for u in frontier:
            for w in adj[u]:
                if w != 7 and w not in dist:
                    dist[w] = dist[u] + 1
                    nxt.append(w)
        frontier = nxt
    for r in (1, 2, 3):
        tau = gauge.spanning_tree(bonds, dims, [12, 13], r, lambda t: t != 7)
        reached = [v for _, v in tau]
        assert len(set(reached)) == len(reached) and not ({12, 13} & set(reached)) and 7 not in reached
        assert all(dist[v] <= r for v in reached)
        region = {12, 13}
        for u, v in tau:
            assert u in region and set(bonds[u]) & set(bonds[v])
            region.add(v)
        ds = [dist[v] for v in reached]
        assert ds == sorted(ds)       # closest first (all bonds have the same size here)
        assert set(reached) == {v for v, d in dist.items() if 0 < d <= r}   # every node within r, once


# ---------------------------------------------------------------------------
# planted mistakes


def test_planted_outward_absorption_breaks_tree_exactness(monkeypatch):
    orig = gauge.spanning_tree
    monkeypatch.setattr(gauge, "spanning_tree", lambda *a, **k: [(v, u) for u, v in orig(*a, **k)])
    net, t = tree_case(1)
    z = approx.contract_exact(net, t)
    try:
        g = gauge.contract_gauged(net, t, 1, 1000, include_inputs=True)
        ok = abs(g.logabs - z.logabs) < 1e-12 * max(1.0, abs(z.logabs))
    except (KeyError, ValueError, IndexError):
        ok = False
    assert not ok


def test_planted_projector_without_inverse_root_breaks_r0_identity(monkeypatch):
    n, e = nw.square_lattice(6, 6)
    net = nw.ising_network(n, e, 0.44)
    tree = tr.boundary_rows(6, 6)
    a = approx.contract(net, tree, 4)          # computed before the mistake is planted
    real_svd = np.linalg.svd

    def svd_squared(m, full_matrices=True):
        u, s, vt = real_svd(m, full_matrices=full_matrices)
        return u, s * s, vt          # the projectors then scale by s^-1 instead of s^-1/2
    monkeypatch.setattr(gauge.np.linalg, "svd", svd_squared)
    g = gauge.contract_gauged(net, tree, 4, 0)
    monkeypatch.undo()
    assert abs(g.logabs - a.logabs) > 1e-6 * abs(a.logabs)
