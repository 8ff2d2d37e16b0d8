"""Span tree builder (Algorithm 2 with r unbounded) and the random-search hyper-optimizer (CPU).

  * Algorithm 2 spans the graph: every node joins once, each pair joins a
    region node to a new neighbour, nodes join in order of distance under the
    default score, and a bounded r stops at that distance;
  * Span trees contract exactly at large chi (transfer matrix, einsum);
  * the GPU executor's schedule for Span trees, early and late, replayed on
    the CPU (tests/plan_emulator.py) matches the oracle at finite chi;
  * the search returns the best traced cost it sampled, and on the 16x16
    D = 4 chi = 64 lattice it beats the boundary-row order.
"""
import numpy as np
import pytest

from oracle import approx, exact
from tn_inputs import networks as nw
from tn_inputs import trees as tr

from plan_emulator import Emulator


def test_local_spanning_tree_properties():
    n, e = nw.square_lattice(5, 6)
    net = nw.random_network(n, e, 2, seed=0)
    tau, order = tr.local_spanning_tree(net.bonds, net.bond_dims, [0])
    assert sorted(order) == list(range(n)) and len(tau) == n - 1
    seen = {0}
    dist = {0: 0}
    for u, v in tau:
        assert u in seen and v not in seen and (v in [o for o in range(n) if set(net.bonds[u]) & set(net.bonds[v])])
        seen.add(v)
        dist[v] = dist[u] + 1
    # default score: closest first, so distances never decrease along the order
    ds = [dist[v] for v in order]
    assert ds == sorted(ds)
    # bounded r: exactly the nodes within graph distance r of the start (manhattan on the grid)
    tau2, order2 = tr.local_spanning_tree(net.bonds, net.bond_dims, [0], r=3)
    assert sorted(order2) == sorted(v for v in range(n) if (v // 5) + (v % 5) <= 3)   # rows of 5 nodes


@pytest.mark.parametrize("start", ["central", "peripheral"])
@pytest.mark.parametrize("policy", ["early", "late"])
def test_span_trees_contract_exactly(start, policy):
    n, e = nw.square_lattice(6, 6)
    net = nw.ising_network(n, e, 0.44)
    t = tr.span(net.bonds, net.bond_dims, policy, start=start)
    got = approx.contract(net, t, 10 ** 6)
    assert abs(got.logabs - exact.ising_transfer_2d(6, 6, 0.44)["lnZ"]) < 1e-12 * got.logabs
    n, e = nw.cubic_lattice(2, 2, 3)
    net = nw.random_network(n, e, 2, seed=4)
    t = tr.span(net.bonds, net.bond_dims, policy, start=start)
    z = exact.einsum_contract(net)
    r = approx.contract_exact(net, t)
    assert r.sign == np.sign(z) and abs(r.logabs - np.log(abs(z))) < 1e-12 * max(1.0, abs(r.logabs))


@pytest.mark.parametrize("policy", ["early", "late"])
def test_gpu_schedule_for_span_trees_replays_to_the_oracle(policy):
    from paper_2206_07044_gb300 import build, tn
    build.build()
    n, e = nw.square_lattice(6, 7)
    net = nw.random_network(n, e, 3, seed=12)
    t = tr.span(net.bonds, net.bond_dims, policy, start="peripheral")
    want = approx.contract(net, t, 6)
    assert want.compressions > 0 and min(d[2] for d in want.diag) > 1e-8
    em = Emulator(tn.plan_describe(net, t, 6), [net]).run()
    assert em.sign[0] == want.sign and abs(em.logabs[0] - want.logabs) <= 1e-10 * abs(want.logabs)


def test_hyper_search_beats_the_boundary_order_on_16x16():
    n, e = nw.square_lattice(16, 16)
    net = nw.random_network(n, e, 4, seed=0)
    tree, params, cost, hist = tr.hyper_search(net.bonds, net.bond_dims, 64, n_trials=64, seed=0)
    assert cost == min(hist)
    assert cost == tr.trace_cost(net.bonds, net.bond_dims, tree, 64)["total"]
    boundary = tr.trace_cost(net.bonds, net.bond_dims, tr.boundary_rows(16, 16), 64)["total"]
    assert cost < boundary, (cost, boundary, params)


# ---------------------------------------------------------------------------
# layer-by-layer boundary order for cubic lattices


def test_boundary_layers_contract_exactly_and_replay():
    n, e = nw.cubic_lattice(3, 2, 3)
    net = nw.random_network(n, e, 2, seed=1)
    t = tr.boundary_layers(3, 2, 3)
    z = exact.einsum_contract(net)
    r = approx.contract_exact(net, t)
    assert r.sign == np.sign(z) and abs(r.logabs - np.log(abs(z))) < 1e-12 * max(1.0, abs(r.logabs))
    from paper_2206_07044_gb300 import build, tn
    build.build()
    n, e = nw.cubic_lattice(3, 3, 3)
    net = nw.ising_network(n, e, 0.5, nw.spin_glass_couplings(len(e), seed=2))
    t = tr.boundary_layers(3, 3, 3)
    want = approx.contract(net, t, 4)
    assert want.compressions > 0 and min(d[2] for d in want.diag) > 1e-8
    em = Emulator(tn.plan_describe(net, t, 4), [net]).run()
    assert em.sign[0] == want.sign and abs(em.logabs[0] - want.logabs) <= 1e-10 * abs(want.logabs)


def test_boundary_layers_make_the_8x8x8_glass_plannable_at_chi_32():
    """8x8x8 +-J glass at chi = 32: a few GB per instance on the layered order
    (the best of 24 sampled Span trees needs about 280 GB)."""
    from paper_2206_07044_gb300 import build, tn
    build.build()
    n, e = nw.cubic_lattice(8, 8, 8)
    net = nw.ising_network(n, e, 0.5, nw.spin_glass_couplings(len(e), seed=0))
    t = tr.boundary_layers(8, 8, 8)
    cost = tr.trace_cost(net.bonds, net.bond_dims, t, 32)
    assert cost["total"] < 1e13 and cost["peak"] < 1e9
    p = tn.plan_describe(net, t, 32)
    assert p["arena_units"] * 8 < 4e9


def test_greedy_with_the_si_input_reduction_stays_near_boundary_rows():
    """Greedy (SI "Greedy") on square lattices, D = 4, chi = 64: with the input sizes
    reduced by their maximum (one of the SI's reductions) the traced cost C stays
    within a small factor of the boundary-row order, while the sum reduction grows
    2D blobs whose tensors explode (the cost C of Sec. "Tree cost functions")."""
    for L, bound in ((16, 6.0), (32, 3.0)):
        n, e = nw.square_lattice(L, L)
        net = nw.random_network(n, e, 4, seed=0)
        base = tr.trace_cost(net.bonds, net.bond_dims, tr.boundary_rows(L, L), 64)["total"]
        g = tr.greedy(net.bonds, net.bond_dims, 64, **tr.greedy_front_params(64))
        c = tr.trace_cost(net.bonds, net.bond_dims, g, 64)
        assert c["total"] < bound * base, (L, c["total"], base)
        if L == 16:
            blob = tr.trace_cost(net.bonds, net.bond_dims, tr.greedy(net.bonds, net.bond_dims, 64), 64)["total"]
            assert blob > 100 * base
