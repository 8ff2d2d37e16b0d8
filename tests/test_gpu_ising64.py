"""The 64 x 64 Ising beta sweep at chi = 128 at full size (GPU), against stored oracle values.

tests/golden/ising64_chi128.json holds the oracle's ln|Z| for six betas of the
sweep beta_t = 0.2 + 0.5 t / 255 (written by tests/golden/make_ising64.py,
which calls only the oracle) together with each value's rounding sensitivity:
the spread of ln|Z| - ln(1 + eps) when one input tensor is scaled by
(1 + eps), |eps| <= 3e-15.  That spread ranges from 4e-12 (beta = 0.7) to
1.2e-5 relative (beta = 0.44, near the critical point), so two correct FP64
implementations can differ by that much end to end; the end-to-end tolerance
at each beta is therefore max(1e-9, 4 x spread) for the FP64 form and
max(1e-6, 4 x spread) for a reduced-precision form (the metric's gate), and
exact parity is checked op by op on two whole boundary rows instead
(tests/oplevel.py).
"""
import json
import os

import numpy as np
import pytest

from tn_inputs import networks as nw
from tn_inputs import trees as tr

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
L, CHI = 64, 128


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "ising64_chi128.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def sweep(golden):
    import torch
    from paper_2206_07044_gb300 import Context, build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    ctx = Context(0)
    n, edges = nw.square_lattice(L, L)
    tree = tr.boundary_rows(L, L)
    ids = [ctx.load_tree(ctx.load_network(nw.ising_network(n, edges, e["beta"])), tree)
           for e in golden["entries"]]
    yield ctx, tree, ids
    ctx.close()


def _band(e, prec):
    # the FP64 form: within the oracle's own rounding band; a reduced-precision
    # form: within the metric's gate of 1e-6, or that band where it is wider
    return max(1e-9 if prec == "f64" else 1e-6, 4.0 * e["spread_rel"])


@pytest.mark.parametrize("prec", ["f64", "tf32x3"])
def test_sweep_end_to_end_within_rounding_band(golden, sweep, prec):
    ctx, tree, ids = sweep
    lz, sg = ctx.contract(ids, CHI, prec)
    errs = []
    for e, got, s in zip(golden["entries"], lz, sg):
        assert s == e["sign"] == 1
        rel = abs(got - e["logabsz"]) / abs(e["logabsz"])
        errs.append(rel)
        assert rel <= _band(e, prec), (prec, e["beta"], got, e["logabsz"], rel, _band(e, prec))
    print(prec, "rel errors vs oracle:", ["%.1e" % x for x in errs])


def test_sweep_rows_match_oracle_op_by_op(sweep):
    """Every C and S op of boundary rows 32 and 63 (the last) for two betas of the batch."""
    from oplevel import row_ops, walk
    ctx, tree, ids = sweep
    ops = [r for y in (32, 63) for r in row_ops(L, y)]
    res = walk(ctx, ids, tree, CHI, ops, (1, 3))
    print("op-level walk:", res)
    assert res["c_ops"] == 2 * 64 * 2
    assert res["s_ops"] + res["ambiguous"] + res["noop"] == 2 * 63 * 2
    assert res["s_ops"] >= 0.8 * (2 * 63 * 2)
