"""Branch-and-bound tree search (SI "Branch & bound approximate contraction tree", CPU).

  * on graphs small enough to enumerate every sequence of adjacent-pair
    contractions (early compression), the search's tree is as cheap as the
    cheapest enumerated one, for the cost C and for the peak memory M, and
    the score it reports is the tracer's value of the tree it returns;
  * seeded with a Greedy tree and stopped early, it returns a tree no worse
    than the seed;
  * its trees contract exactly at large chi.
"""
import math

import numpy as np
import pytest

from oracle import approx, exact
from tn_inputs import networks as nw
from tn_inputs import trees as tr


def _enumerate_min(net, chi, objective):
    """Minimum of the traced objective over every ordered sequence of
    adjacent-pair contractions, each tree built by from_pairs(..., "early")."""
    n = len(net.bonds)
    best = math.inf

    def rec(bonds, pairs, nxt):
        nonlocal best
        live = sorted(bonds)
        if len(live) == 1:
            t = tr.from_pairs(net.bonds, pairs, "early")
            best = min(best, tr.trace_cost(net.bonds, net.bond_dims, t, chi)[objective])
            return
        for x, i in enumerate(live):
            for j in live[x + 1:]:
                if set(bonds[i]) & set(bonds[j]):
                    nb = {k: v for k, v in bonds.items() if k not in (i, j)}
                    si, sj = set(bonds[i]), set(bonds[j])
                    nb[nxt] = [b for b in bonds[i] if b not in sj] + [b for b in bonds[j] if b not in si]
                    rec(nb, pairs + [(i, j)], nxt + 1)

    rec({t: list(b) for t, b in enumerate(net.bonds)}, [], n)
    return best


@pytest.mark.parametrize("objective", ["total", "peak"])
@pytest.mark.parametrize("graph", ["lattice_2x3_d4", "ring5_d5", "k4_d6"])
def test_branch_and_bound_is_optimal_on_enumerable_graphs(graph, objective):
    if graph == "lattice_2x3_d4":
        n, e = nw.square_lattice(2, 3)
        net, chi = nw.random_network(n, e, 4, seed=0), 8
    elif graph == "ring5_d5":
        n, e = nw.ring(5)
        net, chi = nw.random_network(n, e, 5, seed=1), 7
    else:
        n, e = nw.k4()
        net, chi = nw.random_network(n, e, 6, seed=2), 10
    tree, score, complete = tr.branch_and_bound(net.bonds, net.bond_dims, chi, objective)
    assert complete
    assert score == tr.trace_cost(net.bonds, net.bond_dims, tree, chi)[objective]
    assert score == pytest.approx(_enumerate_min(net, chi, objective), rel=1e-12)


def test_branch_and_bound_refines_a_greedy_tree():
    n, e = nw.square_lattice(4, 4)
    net = nw.random_network(n, e, 3, seed=0)
    g = tr.greedy(net.bonds, net.bond_dims, 4)
    gs = tr.trace_cost(net.bonds, net.bond_dims, g, 4)["total"]
    tree, score, complete = tr.branch_and_bound(net.bonds, net.bond_dims, 4, "total", max_nodes=2000, upper=g)
    assert score <= gs and score == tr.trace_cost(net.bonds, net.bond_dims, tree, 4)["total"]
    # the peak-memory search of the same lattice completes and beats Greedy by 2x or more
    tree, score, complete = tr.branch_and_bound(net.bonds, net.bond_dims, 4, "peak", upper=g)
    assert complete and 2 * score <= tr.trace_cost(net.bonds, net.bond_dims, g, 4)["peak"]


def test_branch_and_bound_trees_contract_exactly():
    n, e = nw.square_lattice(3, 3)
    net = nw.ising_network(n, e, 0.44)
    tree, _, complete = tr.branch_and_bound(net.bonds, net.bond_dims, 4, "peak")
    got = approx.contract(net, tree, 10 ** 6)
    assert complete and abs(got.logabs - exact.ising_transfer_2d(3, 3, 0.44)["lnZ"]) < 1e-12 * got.logabs
    n, e = nw.cubic_lattice(2, 2, 2)
    net = nw.random_network(n, e, 2, seed=3)
    tree, _, _ = tr.branch_and_bound(net.bonds, net.bond_dims, 2, "total", max_nodes=5000)
    z = exact.einsum_contract(net)
    r = approx.contract_exact(net, tree)
    assert r.sign == np.sign(z) and abs(r.logabs - np.log(abs(z))) < 1e-12 * max(1.0, abs(r.logabs))
