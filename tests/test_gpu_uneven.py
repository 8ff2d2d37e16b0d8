"""Instances of uneven trees in one call (GPU): random cubic dimer graphs of
different sizes, each with its own Greedy tree, run as concurrent branches of
one pass (and one CUDA graph from the second call on)."""
import math

import numpy as np
import pytest

from oracle import approx, exact
from tn_inputs import networks as nw
from tn_inputs import trees as tr

pytestmark = pytest.mark.gpu


def _ctx(**opt):
    import torch
    from paper_2206_07044_gb300 import Context, build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return Context(0, **opt)


def _graphs(sizes, seed0, chi):
    out = []
    for i, n in enumerate(sizes):
        nv, edges = nw.random_regular_graph(n, 3, seed=seed0 + i)
        net = nw.dimer_network(nv, edges)
        tree = tr.greedy(net.bonds, net.bond_dims, chi=chi, w_inputs=0.0, seed=i)
        out.append((nv, edges, net, tree))
    return out


def _load(c, gs):
    return [c.load_tree(c.load_network(net), tree) for _, _, net, tree in gs]


def test_uneven_small_graphs_exact_matching_counts():
    gs = _graphs([10, 12, 14, 16, 16], 11, 64)
    c = _ctx()
    ids = _load(c, gs)
    for _ in range(3):  # eager, captured, replayed
        lz, sg = c.contract(ids, 64)
        for (nv, edges, _, _), l, s in zip(gs, lz, sg):
            want = exact.perfect_matchings(nv, edges)
            if want == 0:
                assert s == 0 and l == -math.inf
            else:
                assert s == 1 and abs(math.exp(l) - want) < 1e-8 * want
    assert c.graph_info()["captured"] >= 1
    c.close()


def test_uneven_graphs_match_oracle_and_sequential_bitwise():
    gs = _graphs([40, 52, 64, 76, 88, 100], 31, 8)
    c = _ctx()
    ids = _load(c, gs)
    runs = [c.contract(ids, 8)[0] for _ in range(3)]
    c.close()
    assert all(np.array_equal(runs[0], r) for r in runs[1:])
    seq = _ctx(sequential_groups=1)
    sids = _load(seq, gs)
    lz_seq, _ = seq.contract(sids, 8)
    seq.close()
    assert np.array_equal(runs[0], lz_seq)
    checked = 0
    for (_, _, net, tree), l in zip(gs, runs[0]):
        want = approx.contract(net, tree, 8)
        if want.diag and min(d[2] for d in want.diag) <= 1e-8:
            continue  # an ambiguous cut: several truncations are correct
        assert abs(l - want.logabs) <= 1e-10 * abs(want.logabs), (l, want.logabs)
        checked += 1
    assert checked >= 4


def test_split_batch_runs_as_concurrent_sub_batches():
    """tn_options.split_batches = 3: a batch of six instances sharing one tree runs as three
    concurrent sub-batches; the values agree with the unsplit batch and the oracle (16x16
    D=4 chi=64, a well-conditioned case), and the captured pass replays bit for bit."""
    n, e = nw.square_lattice(16, 16)
    tree = tr.boundary_rows(16, 16)
    nets = [nw.random_network(n, e, 4, seed=200 + s) for s in range(6)]
    one = _ctx()
    lz1, _ = one.contract([one.load_tree(one.load_network(x), tree) for x in nets], 64)
    one.close()
    c = _ctx(split_batches=3)
    ids = [c.load_tree(c.load_network(x), tree) for x in nets]
    runs = [c.contract(ids, 64)[0] for _ in range(3)]
    c.close()
    assert all(np.array_equal(runs[0], r) for r in runs[1:])
    for s in (0, 5):
        want = approx.contract(nets[s], tree, 64)
        assert min(d[2] for d in want.diag) > 1e-8
        assert abs(runs[0][s] - want.logabs) <= 1e-10 * abs(want.logabs)
    assert np.all(np.abs(runs[0] - lz1) <= 1e-10 * np.abs(lz1))
