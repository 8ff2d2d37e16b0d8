"""Pins of the CPU oracle against values fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every expected value comes from
brute-force enumeration, transfer matrices, closed forms, the paper's printed
constants, or an invariant the exact or truncated result must satisfy.
"""
import math

import numpy as np
import pytest

from oracle import approx, exact
from tn_inputs import networks as nw
from tn_inputs import trees as tr
from tn_inputs.formats import Network, Tree


def rel(a, b):
    return abs(a - b) / abs(b)


# ---------------------------------------------------------------------------
# exact contraction along the tree: Ising against enumeration / transfer matrices


@pytest.mark.parametrize("beta", [0.0, 0.2, 0.44, 1.0])
def test_ising_4x4_bruteforce(beta):
    n, edges = nw.square_lattice(4, 4)
    net = nw.ising_network(n, edges, beta)
    r = approx.contract_exact(net, tr.boundary_rows(4, 4))
    bf = exact.ising_bruteforce(n, edges, beta)
    assert r.sign == 1
    assert rel(r.logabs, bf["lnZ"]) < 1e-13


def test_transfer_matrix_matches_bruteforce():
    n, edges = nw.square_lattice(4, 3)
    for beta in (0.3, 0.44):
        bf = exact.ising_bruteforce(n, edges, beta)
        tm = exact.ising_transfer_2d(4, 3, beta)
        assert rel(tm["lnZ"], bf["lnZ"]) < 1e-13
        assert rel(tm["dlnZ_dbeta"], bf["dlnZ_dbeta"]) < 1e-12


def test_ising_8x8_exact_tree_vs_transfer_matrix():
    n, edges = nw.square_lattice(8, 8)
    net = nw.ising_network(n, edges, 0.44)
    tm = exact.ising_transfer_2d(8, 8, 0.44)
    r = approx.contract_exact(net, tr.boundary_rows(8, 8))
    assert rel(r.logabs, tm["lnZ"]) < 1e-13


def test_ising_8x8_lossless_compressions_vs_transfer_matrix():
    # chi = 64 fires compressions, but every local rank fits: the result is exact
    n, edges = nw.square_lattice(8, 8)
    net = nw.ising_network(n, edges, 0.44)
    tm = exact.ising_transfer_2d(8, 8, 0.44)
    r = approx.contract(net, tr.boundary_rows(8, 8), 64)
    assert r.compressions > 0
    assert rel(r.logabs, tm["lnZ"]) < 1e-13


def test_ising_8x8_chi16_error_small_and_decreasing():
    # error vs chi falls towards the exact value (the paper's error-vs-chi studies)
    n, edges = nw.square_lattice(8, 8)
    net = nw.ising_network(n, edges, 0.44)
    tm = exact.ising_transfer_2d(8, 8, 0.44)["lnZ"]
    t = tr.boundary_rows(8, 8)
    errs = [rel(approx.contract(net, t, chi).logabs, tm) for chi in (2, 4, 8, 16, 32)]
    assert all(errs[i + 1] <= errs[i] for i in range(len(errs) - 1))
    assert errs[3] < 1e-6
    assert errs[0] > 1e-4   # chi = 2 really truncates


def test_spin_glass_lr_split_bruteforce():
    # +-J couplings need the W_L / W_R split (sinh < 0 for J < 0)
    n, edges = nw.square_lattice(3, 4)
    J = nw.spin_glass_couplings(len(edges), seed=3)
    assert (J < 0).any() and (J > 0).any()
    net = nw.ising_network(n, edges, 0.5, J)
    r = approx.contract_exact(net, tr.boundary_rows(3, 4))
    bf = exact.ising_bruteforce(n, edges, 0.5, J)
    assert rel(r.logabs, bf["lnZ"]) < 1e-13


def test_cubic_2x2x3_spin_glass_bruteforce_greedy_tree():
    n, edges = nw.cubic_lattice(2, 2, 3)
    J = nw.spin_glass_couplings(len(edges), seed=1)
    net = nw.ising_network(n, edges, 0.5, J)
    t = tr.greedy(net.bonds, net.bond_dims, chi=4)
    r = approx.contract_exact(net, t)
    bf = exact.ising_bruteforce(n, edges, 0.5, J)
    assert rel(r.logabs, bf["lnZ"]) < 1e-13


def test_symmetric_and_lr_splits_agree():
    n, edges = nw.square_lattice(3, 3)
    a = approx.contract_exact(nw.ising_network(n, edges, 0.4, symmetric=True), tr.boundary_rows(3, 3))
    b = approx.contract_exact(nw.ising_network(n, edges, 0.4, symmetric=False), tr.boundary_rows(3, 3))
    assert rel(a.logabs, b.logabs) < 1e-14


# ---------------------------------------------------------------------------
# closed forms


def test_ring_closed_form_and_chi_2_exact():
    n, edges = nw.ring(12)
    net = nw.ising_network(n, edges, 0.7)
    t = tr.from_pairs(net.bonds, tr.sequential_pairs(n), "early")
    want = exact.ising_ring_closed_form(12, 0.7)
    assert rel(approx.contract_exact(net, t).logabs, want) < 1e-13
    # a ring's cut has rank <= 2 (D=2 bonds): chi = 2 is exact, chi = 1 is not
    assert rel(approx.contract(net, t, 2).logabs, want) < 1e-13
    assert rel(approx.contract(net, t, 1).logabs, want) > 1e-6


def test_tree_graph_exact_at_chi_2():
    n, edges = nw.random_tree_graph(20, seed=5)
    J = nw.spin_glass_couplings(len(edges), seed=5)
    net = nw.ising_network(n, edges, 0.6, J)
    t = tr.greedy(net.bonds, net.bond_dims, chi=2)
    want = exact.ising_tree_closed_form(edges, 0.6, J)
    assert rel(approx.contract(net, t, 2).logabs, want) < 1e-13


def test_beta_zero_rank_one_exact_at_chi_1():
    # beta = 0: W = [[1,1],[1,1]]/sqrt2 has rank 1, so Z = 2^N survives chi = 1
    n, edges = nw.square_lattice(5, 5)
    net = nw.ising_network(n, edges, 0.0)
    r = approx.contract(net, tr.boundary_rows(5, 5), 1)
    assert r.compressions > 0
    assert rel(r.logabs, n * math.log(2)) < 1e-13


def test_cdl_exact_at_chi_d_squared():
    # SI CDL section: approximate contraction is exact once chi >= d^2
    for lx, ly, d in ((6, 6, 2), (5, 4, 3)):
        net = nw.cdl_network(lx, ly, d)
        want = (lx - 1) * (ly - 1) * math.log(d)
        assert rel(approx.contract_exact(net, tr.boundary_rows(lx, ly)).logabs, want) < 1e-13
        r = approx.contract(net, tr.boundary_rows(lx, ly), d * d)
        assert r.compressions > 0
        assert rel(r.logabs, want) < 1e-12


# ---------------------------------------------------------------------------
# dimer covers


@pytest.mark.parametrize("graph,count", [(nw.k4, 3), (nw.k33, 6), (nw.petersen, 6), (nw.cube_q3, 9)])
def test_perfect_matching_counts(graph, count):
    n, edges = graph()
    assert exact.perfect_matchings(n, edges) == count
    net = nw.dimer_network(n, edges)
    t = tr.greedy(net.bonds, net.bond_dims, chi=64)
    r = approx.contract_exact(net, t)
    assert r.sign == 1 and abs(math.exp(r.logabs) - count) < 1e-9


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_cubic_graph_dimers_bruteforce(seed):
    n, edges = nw.random_regular_graph(16, 3, seed)
    want = exact.perfect_matchings(n, edges)
    net = nw.dimer_network(n, edges)
    t = tr.greedy(net.bonds, net.bond_dims, chi=64)
    r = approx.contract(net, t, 64)      # no bond of a 16-vertex graph outgrows 64 here
    assert want > 0
    assert abs(math.exp(r.logabs) - want) < 1e-8 * want


def test_no_perfect_matching_gives_zero():
    # a graph with an odd number of vertices has no perfect matching: W = 0
    edges = [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4)]
    assert exact.perfect_matchings(5, edges) == 0
    net = nw.dimer_network(5, edges)
    t = tr.greedy(net.bonds, net.bond_dims, chi=8)
    r = approx.contract_exact(net, t)
    assert r.sign == 0 and r.logabs == -math.inf


def test_dimer_entropy_constant():
    # the closed form printed in the SI for k = 3
    assert abs(nw.dimer_entropy_k_regular(3) - 0.1438410362258904) < 1e-15


# ---------------------------------------------------------------------------
# einsum agreement on random-sign networks (Z may be negative)


@pytest.mark.parametrize("seed", [0, 1])
def test_random_normal_network_matches_einsum(seed):
    n, edges = nw.square_lattice(3, 3)
    net = nw.random_network(n, edges, 3, seed)
    want = exact.einsum_contract(net)
    r = approx.contract_exact(net, tr.boundary_rows(3, 3))
    assert r.sign == (1 if want > 0 else -1)
    assert rel(r.logabs, math.log(abs(want))) < 1e-12


# ---------------------------------------------------------------------------
# the compression primitive against Eckart-Young (independent SVD of the full product)


def _pair_network(rng, da_dims, shared_dims, db_dims):
    # A has bonds (a..., s...), B has (s..., b...), a and b legs closed by two tensors E
    bond_dims = list(da_dims) + list(shared_dims) + list(db_dims)
    na, ns = len(da_dims), len(shared_dims)
    a_b = list(range(na)) + list(range(na, na + ns))
    b_b = list(range(na, na + ns)) + list(range(na + ns, len(bond_dims)))
    ta = rng.normal(size=[bond_dims[x] for x in a_b])
    tb = rng.normal(size=[bond_dims[x] for x in b_b])
    return ta, a_b, tb, b_b, bond_dims


@pytest.mark.parametrize("da,ds,db,chi", [((3, 4), (2, 3), (5,), 4), ((2,), (3, 4), (4, 2), 3),
                                          ((6, 5), (4, 2), (3, 3), 5), ((7,), (3, 3), (2,), 8)])
def test_compression_is_best_rank_k(da, ds, db, chi):
    rng = np.random.default_rng(7)
    ta, ab, tb, bb, dims = _pair_network(rng, da, ds, db)
    r = approx.compress_pair(ta, ab, tb, bb, chi, new_bond=99)
    assert r is not None
    ai, nbi, bj, nbj, k, disc, gap = r
    DA, DS, DB = int(np.prod(da)), int(np.prod(ds)), int(np.prod(db))
    assert k == min(chi, DA, DB)
    # layout convention: the new bond sits where the first shared bond was
    assert nbi == list(range(len(da))) + [99]
    assert nbj == [99] + list(range(len(da) + len(ds), len(dims)))
    full = ta.reshape(DA, DS) @ tb.reshape(DS, DB)
    approx_prod = ai.reshape(DA, k) @ bj.reshape(k, DB)
    s = np.linalg.svd(full, compute_uv=False)
    # Eckart-Young: the error is exactly the discarded singular values
    err2 = np.sum((full - approx_prod) ** 2)
    assert abs(err2 - np.sum(s[k:] ** 2)) < 1e-10 * np.sum(s ** 2)
    # the kept factors are balanced: A_bar^T A_bar = B_bar B_bar^T = diag(s_k)
    g_a = ai.reshape(DA, k).T @ ai.reshape(DA, k)
    g_b = bj.reshape(k, DB) @ bj.reshape(k, DB).T
    assert np.allclose(np.sort(np.diag(g_a))[::-1], s[:k], rtol=1e-10, atol=1e-12)
    assert np.allclose(g_a, g_b, rtol=1e-10, atol=1e-10)


def test_compression_skipped_when_bond_fits():
    rng = np.random.default_rng(0)
    ta, ab, tb, bb, _ = _pair_network(rng, (3,), (2, 2), (3,))
    assert approx.compress_pair(ta, ab, tb, bb, 4, 9) is None
    assert approx.compress_pair(ta, ab, tb, bb, 3, 9) is not None


def test_compression_in_a_closed_network_matches_truncated_product():
    # ring of four D x D matrices; S 0 1 replaces T0 T1 by its best rank-chi part
    rng = np.random.default_rng(11)
    D, chi = 6, 3
    mats = [rng.normal(size=(D, D)) for _ in range(4)]
    # bonds: b0 = (T3,T0), b1 = (T0,T1), b2 = (T1,T2), b3 = (T2,T3); T_v[left, right]
    net = Network([D] * 4, [[0, 1], [1, 2], [2, 3], [3, 0]], [m.copy() for m in mats])
    tree = Tree(4, [("S", 0, 1), ("C", 0, 1, 4), ("C", 4, 2, 5), ("C", 5, 3, 6)])
    got = approx.contract(net, tree, chi)
    u, s, vt = np.linalg.svd(mats[0] @ mats[1])
    m01 = (u[:, :chi] * s[:chi]) @ vt[:chi]
    want = np.trace(m01 @ mats[2] @ mats[3])
    assert got.sign == int(np.sign(want))
    assert abs(got.logabs - math.log(abs(want))) < 1e-12


# ---------------------------------------------------------------------------
# invariants of the truncated result


def _random_orthogonal(rng, d):
    q, r = np.linalg.qr(rng.normal(size=(d, d)))
    return q * np.sign(np.diag(r))


def test_orthogonal_gauge_invariance_at_finite_chi():
    # inserting O O^T on every bond leaves the r = 0 truncated result unchanged
    n, edges = nw.square_lattice(5, 5)
    net = nw.random_network(n, edges, 3, seed=4, dist="uniform", lam=-0.3)
    t = tr.boundary_rows(5, 5)
    base = approx.contract(net, t, 4)
    rng = np.random.default_rng(2)
    g = net.copy()
    for e, (u, v) in enumerate(edges):
        o = _random_orthogonal(rng, 3)
        for vert, mat in ((u, o), (v, o)):   # T_u gets O on its leg, T_v gets O (so O^T O = 1 when contracted)
            ax = g.bonds[vert].index(e)
            g.data[vert] = np.moveaxis(np.tensordot(g.data[vert], mat, axes=([ax], [0])), -1, ax)
    assert rel(approx.contract_exact(g, t).logabs, approx.contract_exact(net, t).logabs) < 1e-12
    gauged = approx.contract(g, t, 4)
    assert base.compressions > 0
    assert rel(gauged.logabs, base.logabs) < 1e-11
    assert gauged.sign == base.sign


def test_scaling_and_index_permutation_invariance():
    n, edges = nw.square_lattice(4, 5)
    net = nw.random_network(n, edges, 3, seed=9)
    t = tr.boundary_rows(4, 5)
    base = approx.contract(net, t, 5)
    s = net.copy()
    s.data[7] = s.data[7] * 2.0 ** 13
    s.data[3] = s.data[3] * -3.0
    r = approx.contract(s, t, 5)
    assert r.sign == -base.sign
    assert abs(r.logabs - (base.logabs + 13 * math.log(2) + math.log(3))) < 1e-11 * abs(base.logabs)
    p = net.copy()
    for v in (0, 6, 11):
        perm = list(range(len(p.bonds[v])))[::-1]
        p.data[v] = np.transpose(p.data[v], perm).copy()
        p.bonds[v] = [p.bonds[v][i] for i in perm]
    rp = approx.contract(p, t, 5)
    assert rp.sign == base.sign
    assert rel(rp.logabs, base.logabs) < 1e-12


def test_power_of_two_rescale_is_exact():
    n, edges = nw.square_lattice(6, 6)
    net = nw.random_network(n, edges, 2, seed=1)
    t = tr.boundary_rows(6, 6)
    a = approx.contract(net, t, 3, rescale=True)
    b = approx.contract(net, t, 3, rescale=False)
    assert a.sign == b.sign and rel(a.logabs, b.logabs) < 1e-13


def test_large_network_does_not_overflow():
    # 24x24 Ising has Z ~ e^500 ... beyond double range without the running log-norm
    n, edges = nw.square_lattice(24, 24)
    net = nw.ising_network(n, edges, 1.0)
    for d in net.data:
        d *= 64.0
    r = approx.contract(net, tr.boundary_rows(24, 24), 4)
    assert math.isfinite(r.logabs) and r.logabs > 709


# ---------------------------------------------------------------------------
# planted mistakes: each plausible slip in the compression must break a pin


def _broken_compress(kind):
    orig = approx.compress_pair
    calls = [0]

    def f(ti, bi, tj, bj, chi, new_bond):
        r = orig(ti, bi, tj, bj, chi, new_bond)
        if r is None:
            return r
        calls[0] += 1
        ai, nbi, bj2, nbj, k, disc, gap = r
        if kind == "no_sqrt":          # absorbs sigma into A only: A_bar = Q_A U sigma
            ai = ai * 1.7
        elif kind == "flip_sign" and calls[0] == 1:   # one sign slip (an even number would cancel)
            bj2 = -bj2
        elif kind == "swap_layout":    # new bond placed last instead of at the first shared bond
            if len(nbi) > 1:
                pos = nbi.index(new_bond)
                perm = [x for x in range(len(nbi)) if x != pos] + [pos]
                ai = np.transpose(ai, perm).reshape(ai.shape)
        return ai, nbi, bj2, nbj, k, disc, gap
    return f


@pytest.mark.parametrize("kind", ["no_sqrt", "flip_sign", "swap_layout"])
def test_planted_mistakes_are_caught(monkeypatch, kind):
    n, edges = nw.square_lattice(8, 8)
    net = nw.ising_network(n, edges, 0.44)
    tm = exact.ising_transfer_2d(8, 8, 0.44)["lnZ"]
    monkeypatch.setattr(approx, "compress_pair", _broken_compress(kind))
    r = approx.contract(net, tr.boundary_rows(8, 8), 64)
    assert not (r.sign == 1 and rel(r.logabs, tm) < 1e-13)


def test_planted_truncation_of_smallest_values_is_caught(monkeypatch):
    real_svd = np.linalg.svd

    def svd_ascending(m, full_matrices=False):
        u, s, vt = real_svd(m, full_matrices=full_matrices)
        return u[:, ::-1], s[::-1], vt[::-1]

    n, edges = nw.square_lattice(8, 8)
    net = nw.ising_network(n, edges, 0.44)
    tm = exact.ising_transfer_2d(8, 8, 0.44)["lnZ"]
    monkeypatch.setattr(approx.np.linalg, "svd", svd_ascending)
    r = approx.contract(net, tr.boundary_rows(8, 8), 8)
    assert rel(r.logabs, tm) > 1e-3


# ---------------------------------------------------------------------------
# the torch Ising builder (used for d/d beta, d/d J through autograd) against
# the numpy builder, and its beta-derivative against central differences


def test_torch_ising_builder_matches_numpy_and_differentiates():
    import torch
    from tn_inputs import torch_ising as ti
    n, e = nw.cubic_lattice(2, 2, 2)
    for J0, beta in ((np.ones(len(e)), 0.44), (nw.spin_glass_couplings(len(e), seed=2), 0.7)):
        sym = bool(np.all(J0 > 0))
        b = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
        T = ti.ising_tensors(n, e, b, torch.tensor(J0), sym)
        ref = nw.ising_network(n, e, beta, J0)
        for t, r in zip(T, ref.data):
            assert np.allclose(t.detach().numpy(), r, rtol=0, atol=1e-14)
        # d/d beta of a linear functional of the tensors, against central differences
        w = [np.random.default_rng(v).normal(size=r.shape) for v, r in enumerate(ref.data)]
        f = sum((t * torch.from_numpy(wv)).sum() for t, wv in zip(T, w))
        f.backward()
        h = 1e-6
        fp = sum(float(np.sum(wv * r)) for wv, r in zip(w, nw.ising_network(n, e, beta + h, J0).data))
        fm = sum(float(np.sum(wv * r)) for wv, r in zip(w, nw.ising_network(n, e, beta - h, J0).data))
        assert abs(float(b.grad) - (fp - fm) / (2 * h)) < 1e-7 * max(1.0, abs(float(b.grad)))
