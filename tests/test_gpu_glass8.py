"""The 8 x 8 x 8 +-J spin glass at chi = 32 at full size (GPU), against stored oracle values.

tests/golden/glass8_chi32.json holds the oracle's ln|Z| for two coupling seeds
(beta = 0.5, the layer-by-layer boundary tree; written by
tests/golden/make_glass8.py, which calls only the oracle) with each value's
spread under 1e-15 relative perturbations of one input.  Checked here: the
FP64 form within max(1e-10, 4 x spread) (the stored spread is at rounding level: this
workload is well conditioned), the BF16 form (contraction GEMMs in
BF16 with FP32 accumulation, QR and SVD in FP64) within the BF16 unit
roundoff, and d ln Z / d J_ij through the reverse pass (tn_grad and the torch
builder) against central differences of the GPU's own FP64 form on four
seeded couplings.
"""
import json
import os

import numpy as np
import pytest

from tn_inputs import networks as nw
from tn_inputs import trees as tr

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
L, CHI, BETA = 8, 32, 0.5


@pytest.fixture(scope="module")
def golden():
    path = os.path.join(HERE, "golden", "glass8_chi32.json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle values")
    with open(path) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def glass(golden):
    import torch
    from paper_2206_07044_gb300 import Context, build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    ctx = Context(0)
    n, edges = nw.cubic_lattice(L, L, L)
    tree = tr.boundary_layers(L, L, L)
    ids = [ctx.load_tree(ctx.load_network(nw.ising_network(n, edges, BETA, nw.spin_glass_couplings(len(edges), e["seed"]))),
                         tree) for e in golden["entries"]]
    yield ctx, n, edges, tree, ids
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "bf16"])
def test_glass_end_to_end(golden, glass, prec):
    ctx, n, edges, tree, ids = glass
    lz, sg = ctx.contract(ids, CHI, prec)
    for e, got, s in zip(golden["entries"], lz, sg):
        tol = max(1e-10, 4 * e["spread_rel"]) if prec == "f64" else max(2.0 ** -8, 4 * e["spread_rel"])
        rel = abs(got - e["logabsz"]) / abs(e["logabsz"])
        print(prec, e["seed"], got, e["logabsz"], "%.2e" % rel)
        assert s == e["sign"] and rel <= tol, (prec, e["seed"], rel, tol)


def test_glass_coupling_gradient_vs_central_differences(golden, glass):
    import torch
    from paper_2206_07044_gb300.autograd import log_z
    from tn_inputs import torch_ising as ti
    ctx, n, edges, tree, ids = glass
    J0 = nw.spin_glass_couplings(len(edges), golden["entries"][0]["seed"])
    J = torch.tensor(J0, dtype=torch.float64, requires_grad=True)
    T = ti.ising_tensors(n, edges, torch.tensor(BETA, dtype=torch.float64), J, False)
    lz = log_z(ctx, ids[0], T, CHI)
    lz.backward()
    g = J.grad.numpy()
    rng = np.random.default_rng(5)
    pick = rng.choice(len(edges), size=4, replace=False)
    h = 1e-5
    fd_ctx_net = ctx._inst_net[ids[0]]
    for k in pick:
        vals = []
        for sgn in (1, -1):
            Jk = J0.copy()
            Jk[k] += sgn * h
            net = nw.ising_network(n, edges, BETA, Jk)
            ctx.set_network_data(fd_ctx_net, net.data)
            vals.append(float(ctx.contract([ids[0]], CHI)[0][0]))
        fd = (vals[0] - vals[1]) / (2 * h)
        print("coupling", k, "reverse pass", g[k], "central difference", fd)
        assert abs(g[k] - fd) <= 1e-4 * max(1.0, abs(fd)), (k, g[k], fd)
    net0 = nw.ising_network(n, edges, BETA, J0)
    ctx.set_network_data(fd_ctx_net, net0.data)
