"""Pins of the oracle's reverse pass (d log|Z| / d T_v) against independent truths.

  * central finite differences of the oracle's forward contraction
    (oracle.approx, a different code path: QR/LQ and the SVD of the core);
  * Euler's identity: the approximate contraction is positively homogeneous of
    degree 1 in each input (contractions multiply scales, compressions split a
    scale c into c^1/2 on each side), so sum(T_v * dlog|Z|/dT_v) = 1 for every
    v at any chi;
  * exact derivatives: with no truncation, dZ/dT_v is the contraction of the
    network with T_v removed (numpy einsum); d ln Z / d beta of the Ising model
    from brute-force enumeration, the row transfer matrix and the ring's closed
    form (the chain rule through the site tensors uses central differences of
    the tensor builder in beta).
Planted mistakes in the SVD adjoint must break the finite-difference pin.
"""
import math

import numpy as np
import pytest

from oracle import approx, exact, grad
from tn_inputs import networks as nw
from tn_inputs import trees as tr
from tn_inputs.formats import Network


def fd_worst(net, tree, chi, g, n_samples=12, h=1e-4, seed=0):
    """Largest |central FD - gradient| over sampled entries, relative to max |gradient|."""
    rng = np.random.default_rng(seed)
    gmax = max(float(np.max(np.abs(x))) for x in g.grads)
    worst = 0.0
    for _ in range(n_samples):
        v = int(rng.integers(net.n_tensors))
        idx = tuple(int(rng.integers(s)) for s in net.data[v].shape)
        vals = []
        for sgn in (1, -1):
            d = [x.copy() for x in net.data]
            d[v][idx] += sgn * h
            vals.append(approx.contract(Network(net.bond_dims, net.bonds, d), tree, chi).logabs)
        fd = (vals[0] - vals[1]) / (2 * h)
        worst = max(worst, abs(fd - g.grads[v][idx]) / gmax)
    return worst


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
    return out


CASES = cases()


@pytest.mark.parametrize("name,net,tree,chi", CASES, ids=[c[0] for c in CASES])
def test_grad_matches_central_differences(name, net, tree, chi):
    g = grad.contract_with_grad(net, tree, chi)
    assert g.compressions > 0, "the case must truncate"
    assert g.min_gap > 1e-3, "truncation must be unambiguous"
    assert g.min_kept > 1e-6, "a kept singular value is zero: not differentiable there"
    assert fd_worst(net, tree, chi, g) < 1e-6


@pytest.mark.parametrize("name,net,tree,chi", CASES, ids=[c[0] for c in CASES])
def test_grad_euler_identity_and_forward(name, net, tree, chi):
    g = grad.contract_with_grad(net, tree, chi)
    want = approx.contract(net, tree, chi)
    assert g.sign == want.sign and abs(g.logabs - want.logabs) < 1e-12 * abs(want.logabs)
    for t, gv in zip(net.data, g.grads):
        assert abs(float(np.sum(t * gv)) - 1.0) < 1e-11


def test_exact_mode_gradient_is_environment_contraction():
    n, e = nw.square_lattice(3, 3)
    net = nw.random_network(n, e, 2, seed=7)
    g = grad.contract_with_grad(net, tr.boundary_rows(3, 3), None)
    z = exact.einsum_contract(net)
    letters = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"
    for v in (0, 4, 8):
        terms, ops = [], []
        for w in range(net.n_tensors):
            if w != v:
                terms.append("".join(letters[b] for b in net.bonds[w]))
                ops.append(net.data[w])
        env = np.einsum(",".join(terms) + "->" + "".join(letters[b] for b in net.bonds[v]), *ops)
        assert np.allclose(g.grads[v], env / z, rtol=1e-12, atol=1e-13 * np.max(np.abs(env / z)))


def dlnz_dbeta(build, beta, tree, chi, h=1e-6):
    """sum_v <d log|Z|/d T_v, d T_v / d beta>, with dT/dbeta by central differences of the builder."""
    g = grad.contract_with_grad(build(beta), tree, chi)
    tp, tm = build(beta + h), build(beta - h)
    return g.logabs, sum(float(np.sum(gv * (a - b) / (2 * h))) for gv, a, b in zip(g.grads, tp.data, tm.data))


def test_dlnz_dbeta_bruteforce_4x4():
    n, e = nw.square_lattice(4, 4)
    lz, d = dlnz_dbeta(lambda b: nw.ising_network(n, e, b), 0.44, tr.boundary_rows(4, 4), 64)
    bf = exact.ising_bruteforce(n, e, 0.44)
    assert abs(lz - bf["lnZ"]) < 1e-12 * lz
    assert abs(d - bf["dlnZ_dbeta"]) < 1e-8 * abs(bf["dlnZ_dbeta"])


def test_dlnz_dbeta_transfer_matrix_8x8():
    n, e = nw.square_lattice(8, 8)
    lz, d = dlnz_dbeta(lambda b: nw.ising_network(n, e, b), 0.44, tr.boundary_rows(8, 8), None)
    tm = exact.ising_transfer_2d(8, 8, 0.44)
    assert abs(lz - tm["lnZ"]) < 1e-12 * lz
    assert abs(d - tm["dlnZ_dbeta"]) < 1e-9 * abs(tm["dlnZ_dbeta"])


def test_dlnz_dbeta_ring_closed_form():
    n, e = nw.ring(12)
    build = lambda b: nw.ising_network(n, e, b)
    lz, d = dlnz_dbeta(build, 0.6, tr.from_pairs(build(0.6).bonds, tr.sequential_pairs(n), "early"), None)
    c, s_ = math.cosh(0.6), math.sinh(0.6)
    z = (2 * c) ** 12 + (2 * s_) ** 12
    want = 12 * ((2 * c) ** 11 * 2 * s_ + (2 * s_) ** 11 * 2 * c) / z
    assert abs(lz - math.log(z)) < 1e-13 * lz
    assert abs(d - want) < 1e-9 * abs(want)


def test_dlnz_dbeta_ising_8x8_chi16_matches_fd_of_forward():
    """The configuration with 18 compressions: the beta-derivative through the
    reverse pass against central differences of the forward oracle in beta."""
    n, e = nw.square_lattice(8, 8)
    build = lambda b: nw.ising_network(n, e, b)
    tree = tr.boundary_rows(8, 8)
    lz, d = dlnz_dbeta(build, 0.44, tree, 16)
    h = 1e-5
    fd = (approx.contract(build(0.44 + h), tree, 16).logabs - approx.contract(build(0.44 - h), tree, 16).logabs) / (2 * h)
    assert abs(d - fd) < 1e-6 * abs(fd)


# ---------------------------------------------------------------------------
# planted mistakes in the SVD adjoint must be caught


def _planted(kind):
    orig = grad.svd_truncated_adjoint

    def bad(u, s, vt, k, ab, bb):
        if kind == "no_complement":
            # both (1 - U U^T) terms dropped: same as projecting the incoming adjoints onto U, V
            return orig(u, s, vt, k, u @ (u.T @ ab), (bb @ vt.T) @ vt)
        if kind == "drop_bbar":
            # the B_bar side of the adjoint forgotten
            return orig(u, s, vt, k, ab, np.zeros_like(bb))
        raise ValueError(kind)
    return bad


@pytest.mark.parametrize("kind", ["no_complement", "drop_bbar", "broad_eps"])
def test_planted_adjoint_mistakes_fail_fd(monkeypatch, kind):
    name, net, tree, chi = CASES[2]
    if kind == "broad_eps":
        monkeypatch.setattr(grad, "EPS_REL", 1e-2)     # broadening far wider than the gaps
    else:
        monkeypatch.setattr(grad, "svd_truncated_adjoint", _planted(kind))
    g = grad.contract_with_grad(net, tree, chi)
    assert fd_worst(net, tree, chi, g) > 1e-4
