"""GPU reverse pass (tn_grad) against the oracle's reverse pass and exact derivatives.

Element-wise parity: max |g_gpu - g_oracle| <= GRAD_TOL * max |g_oracle| on
cases whose truncation is unambiguous and whose kept singular values are well
away from zero (the same cases the oracle is pinned on).  The SVD adjoint
multiplies rounding differences of the forward pass by up to s_1^2 / (s_i^2 -
s_j^2); with relative gaps >= 1e-3 and FP64 forward agreement near 1e-14 that
bounds the difference near 1e-8, the tolerance used here.  At full size the
gradient is checked through Euler's identity, sum(T_v * g_v) = 1 for every
input v, which holds at any chi.
"""
import math

import numpy as np
import pytest

from oracle import approx, exact, grad
from tn_inputs import networks as nw
from tn_inputs import trees as tr

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-8


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2206_07044_gb300 import build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    from paper_2206_07044_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def gpu_grad(ctx, net, tree, chi, prec="f64"):
    iid = ctx.load_tree(ctx.load_network(net), tree)
    lz, sg, g = ctx.grad([iid], chi, prec)
    return float(lz[0]), int(sg[0]), g[0]


def max_rel(ga, gb):
    scale = max(float(np.max(np.abs(x))) for x in gb)
    return max(float(np.max(np.abs(a - b))) for a, b in zip(ga, gb)) / scale


def cases():
    out = []
    n, e = nw.square_lattice(4, 4)
    out.append(("ising 4x4 chi2", nw.ising_network(n, e, 0.44), tr.boundary_rows(4, 4), 2))
    out.append(("normal 4x4 D2 chi3", nw.random_network(n, e, 2, seed=1), tr.boundary_rows(4, 4), 3))
    n, e = nw.square_lattice(5, 4)
    net = nw.random_network(n, e, 3, seed=2)
    out.append(("normal 5x4 D3 chi4 greedy", net, tr.greedy(net.bonds, net.bond_dims, chi=4, seed=0), 4))
    n, e = nw.cubic_lattice(2, 2, 3)
    J = nw.spin_glass_couplings(len(e), seed=0)
    net = nw.ising_network(n, e, 0.5, J)
    out.append(("spin glass 2x2x3 chi2", net, tr.greedy(net.bonds, net.bond_dims, chi=2, seed=1), 2))
    n, e = nw.square_lattice(5, 4)
    net = nw.random_network(n, e, 3, seed=7, dist="uniform", lam=-0.2)
    out.append(("uniform 5x4 late tree", net, tr.from_pairs(net.bonds, tr.sequential_pairs(n), "late"), 2))
    n, e = nw.square_lattice(6, 6)
    out.append(("normal 6x6 D3 chi5", nw.random_network(n, e, 3, seed=3), tr.boundary_rows(6, 6), 5))
    return out


CASES = cases()


@pytest.mark.parametrize("name,net,tree,chi", CASES, ids=[c[0] for c in CASES])
def test_grad_matches_oracle(ctx, name, net, tree, chi):
    want = grad.contract_with_grad(net, tree, chi)
    assert want.min_gap > 1e-3 and want.min_kept > 1e-6
    lz, sg, g = gpu_grad(ctx, net, tree, chi)
    assert sg == want.sign and abs(lz - want.logabs) <= 1e-10 * abs(want.logabs)
    err = max_rel(g, want.grads)
    print(f"grad parity {name}: {err:.2e}")
    assert err <= GRAD_TOL, (name, err)


def test_grad_euler_identity_16x16_d4_chi64(ctx):
    """The shapes of the full workload (compressions of 256-wide cores), checked by homogeneity."""
    n, e = nw.square_lattice(16, 16)
    net = nw.random_network(n, e, 4, seed=0)
    lz, sg, g = gpu_grad(ctx, net, tr.boundary_rows(16, 16), 64)
    want = approx.contract(net, tr.boundary_rows(16, 16), 64)
    assert sg == want.sign and abs(lz - want.logabs) <= 1e-10 * abs(want.logabs)
    worst = max(abs(float(np.sum(t * gv)) - 1.0) for t, gv in zip(net.data, g))
    print(f"euler 16x16: {worst:.2e}")
    assert worst < 1e-8, worst


def test_dlnz_dbeta_exact_vs_transfer_matrix(ctx):
    """No truncation (chi above every bond): d ln Z / d beta of the 8x8 Ising model is exact."""
    import torch
    from paper_2206_07044_gb300.autograd import log_z
    from tn_inputs import torch_ising as ti
    n, e = nw.square_lattice(8, 8)
    net = nw.ising_network(n, e, 0.44)
    iid = ctx.load_tree(ctx.load_network(net), tr.boundary_rows(8, 8))
    beta = torch.tensor(0.44, dtype=torch.float64, requires_grad=True)
    T = ti.ising_tensors(n, e, beta, torch.ones(len(e), dtype=torch.float64), True)
    lz = log_z(ctx, iid, T, 1024)
    lz.backward()
    tm = exact.ising_transfer_2d(8, 8, 0.44)
    assert abs(float(lz.detach()) - tm["lnZ"]) < 1e-12 * tm["lnZ"]
    assert abs(float(beta.grad) - tm["dlnZ_dbeta"]) < 1e-9 * abs(tm["dlnZ_dbeta"])


def test_dlnz_dbeta_config_8x8_chi16(ctx):
    """The 18-compression configuration: d ln Z / d beta through the GPU reverse pass
    against the oracle's reverse pass and against central differences of the oracle."""
    import torch
    from paper_2206_07044_gb300.autograd import log_z
    from tn_inputs import torch_ising as ti
    n, e = nw.square_lattice(8, 8)
    tree = tr.boundary_rows(8, 8)
    iid = ctx.load_tree(ctx.load_network(nw.ising_network(n, e, 0.44)), tree)
    beta = torch.tensor(0.44, dtype=torch.float64, requires_grad=True)
    T = ti.ising_tensors(n, e, beta, torch.ones(len(e), dtype=torch.float64), True)
    lz = log_z(ctx, iid, T, 16)
    lz.backward()
    d_gpu = float(beta.grad)
    # oracle: the same chain rule with the oracle's tensor gradients
    g = grad.contract_with_grad(nw.ising_network(n, e, 0.44), tree, 16)
    Td = [t.detach() for t in T]
    beta2 = torch.tensor(0.44, dtype=torch.float64, requires_grad=True)
    T2 = ti.ising_tensors(n, e, beta2, torch.ones(len(e), dtype=torch.float64), True)
    torch.autograd.backward(T2, [torch.from_numpy(x) for x in g.grads])
    assert abs(d_gpu - float(beta2.grad)) < 1e-8 * abs(d_gpu)
    h = 1e-5
    fd = (approx.contract(nw.ising_network(n, e, 0.44 + h), tree, 16).logabs -
          approx.contract(nw.ising_network(n, e, 0.44 - h), tree, 16).logabs) / (2 * h)
    assert abs(d_gpu - fd) < 1e-6 * abs(fd)
    assert Td[0].shape == T[0].shape


def test_dlnz_dcouplings_spin_glass(ctx):
    """d ln Z / d J_ij of a cubic +-J glass through the GPU reverse pass vs central differences (h=1e-5)."""
    import torch
    from paper_2206_07044_gb300.autograd import log_z
    from tn_inputs import torch_ising as ti
    n, e = nw.cubic_lattice(2, 2, 3)
    J0 = nw.spin_glass_couplings(len(e), seed=0)
    net = nw.ising_network(n, e, 0.5, J0)
    tree = tr.greedy(net.bonds, net.bond_dims, chi=2, seed=1)
    iid = ctx.load_tree(ctx.load_network(net), tree)
    J = torch.tensor(J0, dtype=torch.float64, requires_grad=True)
    T = ti.ising_tensors(n, e, torch.tensor(0.5, dtype=torch.float64), J, False)
    lz = log_z(ctx, iid, T, 2)
    lz.backward()
    h = 1e-5
    for k in range(0, len(e), 3):
        Jp, Jm = J0.copy(), J0.copy()
        Jp[k] += h
        Jm[k] -= h
        fd = (approx.contract(nw.ising_network(n, e, 0.5, Jp), tree, 2).logabs -
              approx.contract(nw.ising_network(n, e, 0.5, Jm), tree, 2).logabs) / (2 * h)
        assert abs(float(J.grad[k]) - fd) < 1e-6 * max(1.0, abs(fd)), (k, float(J.grad[k]), fd)


def test_grad_batched_matches_individual_and_replays(ctx):
    n, e = nw.square_lattice(6, 6)
    tree = tr.boundary_rows(6, 6)
    nets = [nw.random_network(n, e, 3, seed=10 + s) for s in range(3)]
    ids = [ctx.load_tree(ctx.load_network(x), tree) for x in nets]
    lz, sg, g = ctx.grad(ids, 5)
    lz2, sg2, g2 = ctx.grad(ids, 5)   # captured as a graph
    lz3, sg3, g3 = ctx.grad(ids, 5)   # replayed
    for a, b, c in zip(g, g2, g3):
        for x, y, z in zip(a, b, c):
            assert np.array_equal(x, y) and np.array_equal(x, z)
    for s, x in enumerate(nets):
        want = grad.contract_with_grad(x, tree, 5)
        if want.min_gap > 1e-3 and want.min_kept > 1e-6:
            assert max_rel(g[s], want.grads) <= GRAD_TOL
        one = ctx.grad([ids[s]], 5)
        assert max_rel(one[2][0], g[s]) <= 1e-12


def test_grad_mixed_form_close_to_f64(ctx):
    """Split-TF32 contraction GEMMs in both passes, on a well-conditioned case (cut gaps
    >= 1e-3 s_1, kept values >= 1e-6 s_1): the gradient stays within FP32 roundoff
    (2^-24) times the adjoint's 1/gap amplification, bounded here by 1e-4 of max |g|.
    (On cases with near-degenerate cuts, such as the 8x8 Ising chi=16 configuration
    whose cut gaps reach 2e-13, any rounding is amplified without bound.)"""
    name, net, tree, chi = CASES[-1]
    want = grad.contract_with_grad(net, tree, chi)
    assert want.min_gap > 1e-3 and want.min_kept > 1e-6
    _, _, g64 = gpu_grad(ctx, net, tree, chi)
    _, _, g3 = gpu_grad(ctx, net, tree, chi, "tf32x3")
    err = max_rel(g3, g64)
    print(f"tf32x3 gradient vs f64: {err:.2e}")
    assert err <= 1e-4, err


def test_grad_of_zero_partition_function_is_an_error(ctx):
    from paper_2206_07044_gb300 import TNError
    edges = [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4)]
    net = nw.dimer_network(5, edges)
    with pytest.raises(TNError) as ei:
        gpu_grad(ctx, net, tr.greedy(net.bonds, net.bond_dims, chi=8), 8)
    assert ei.value.code == -7


def test_grad_checkpointed_equals_one_tape(ctx):
    """Checkpointed reverse pass (3 segments): the recomputation repeats the same kernels on
    the same data, so the gradient equals the one-tape pass."""
    n, e = nw.square_lattice(6, 6)
    net = nw.random_network(n, e, 3, seed=3)
    tree = tr.boundary_rows(6, 6)
    iid = ctx.load_tree(ctx.load_network(net), tree)
    ctx.set_grad_segments(1)
    lz1, _, g1 = ctx.grad([iid], 5)
    ctx.set_grad_segments(3)
    lz3, _, g3 = ctx.grad([iid], 5)
    ctx.set_grad_segments(0)
    assert lz1[0] == lz3[0]
    assert max_rel(g3[0], g1[0]) <= 1e-13
    want = grad.contract_with_grad(net, tree, 5)
    assert max_rel(g3[0], want.grads) <= GRAD_TOL


def test_dlnz_dbeta_batched_sweep(ctx):
    """Internal energy of a beta sweep from one tn_grad call (log_z_batch) equals the
    per-instance wrapper and the oracle's reverse pass at every beta."""
    import torch
    from paper_2206_07044_gb300.autograd import log_z, log_z_batch
    from tn_inputs import torch_ising as ti
    n, e = nw.square_lattice(8, 8)
    tree = tr.boundary_rows(8, 8)
    betas = [0.3, 0.41, 0.44, 0.52, 0.65]
    ids = [ctx.load_tree(ctx.load_network(nw.ising_network(n, e, b)), tree) for b in betas]
    bt = [torch.tensor(b, dtype=torch.float64, requires_grad=True) for b in betas]
    ones = torch.ones(len(e), dtype=torch.float64)
    lz = log_z_batch(ctx, ids, [ti.ising_tensors(n, e, b, ones, True) for b in bt], 16)
    assert lz.shape == (len(betas),)
    lz.sum().backward()
    for b, iid, bb, l in zip(betas, ids, bt, lz.detach()):
        b1 = torch.tensor(b, dtype=torch.float64, requires_grad=True)
        l1 = log_z(ctx, iid, ti.ising_tensors(n, e, b1, ones, True), 16)
        l1.backward()
        assert abs(float(l) - float(l1)) <= 1e-13 * abs(float(l1))
        assert abs(float(bb.grad) - float(b1.grad)) <= 1e-10 * abs(float(b1.grad))
        g = grad.contract_with_grad(nw.ising_network(n, e, b), tree, 16)
        b2 = torch.tensor(b, dtype=torch.float64, requires_grad=True)
        T2 = ti.ising_tensors(n, e, b2, ones, True)
        torch.autograd.backward(T2, [torch.from_numpy(x) for x in g.grads])
        assert abs(float(bb.grad) - float(b2.grad)) < 1e-8 * abs(float(b2.grad))
