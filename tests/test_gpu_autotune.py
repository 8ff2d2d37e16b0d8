"""The launch-shape autotuner (GPU): tuned shapes keep results exact and round-trip
through the cache file."""
import os

import pytest

from oracle import approx
from tn_inputs import networks as nw
from tn_inputs import trees as tr

pytestmark = pytest.mark.gpu

FAMILIES = {1: "qr", 2: "jacobi_f64", 3: "jacobi_f32", 4: "gemm_f64", 5: "gemm_tc"}


def _ctx(**opt):
    import torch
    from paper_2206_07044_gb300 import Context, build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return Context(0, **opt)


def test_autotune_choices_valid_results_exact_and_cached(tmp_path):
    cache = str(tmp_path / "tune.txt")
    c = _ctx(tuner_cache=cache)
    n, e = nw.square_lattice(12, 12)
    tree = tr.boundary_rows(12, 12)
    nets = [nw.random_network(n, e, 4, seed=s) for s in range(3)]
    ids = [c.load_tree(c.load_network(x), tree) for x in nets]
    before, _ = c.contract(ids, 32)
    tuned = c.autotune(ids, 32)
    assert tuned > 0
    rows = c.tuned_choices()
    fams = {r[0] for r in rows if r[4] == 3}
    assert {1, 2, 3, 4} <= fams, rows
    for fam, m, nn, k, batch, val in rows:
        assert fam in FAMILIES and m > 0 and nn > 0 and batch > 0
        if fam in (1, 2, 3):
            assert 1 <= val <= 16
        elif fam == 4:
            assert 1 <= val <= 4
    after, _ = c.contract(ids, 32)
    for s, x in enumerate(nets):
        want = approx.contract(x, tree, 32)
        assert min(d[2] for d in want.diag) > 1e-8
        assert abs(after[s] - want.logabs) <= 1e-10 * abs(want.logabs)
        assert abs(before[s] - want.logabs) <= 1e-10 * abs(want.logabs)
    c.close()
    assert os.path.exists(cache)
    head = open(cache).readline().split()
    assert head[:2] == ["tntune", "1"]
    # a new context reads the cache back
    c2 = _ctx(tuner_cache=cache)
    assert sorted(c2.tuned_choices()) == sorted(rows)
    c2.close()
