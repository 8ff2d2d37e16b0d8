"""The library's schedules, replayed on the CPU, against the oracle (host logic, no GPU).

`tn_plan_describe` exports the exact step list the GPU executor runs
(schedule expansion of Algorithm 1, the static arena, operand orientations,
the reverse pass of tn_grad); `plan_emulator` replays it in numpy with the
executor's buffer layout.  Results must match the oracle: log|Z| to 1e-10
relative (every form's schedule, emulated in FP64), gradients to 1e-8 of
max |g| on the oracle's pinned cases.  Planted planner-style mistakes in an
exported schedule (a transposed operand view, a wrong rescale slot, a
dropped reverse step) must make the replay disagree.
"""
import copy
import math

import numpy as np
import pytest

from oracle import approx, grad
from tn_inputs import networks as nw
from tn_inputs import trees as tr

from plan_emulator import Emulator, ST_GEMM, ST_SCALE_POW2, ST_SVD_ADJ_CORE

TOL = 1e-10
GRAD_TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_07044_gb300 import build
    build.build()


def describe(net, tree, chi, prec="f64", g=False):
    from paper_2206_07044_gb300 import tn
    return tn.plan_describe(net, tree, chi, prec, g)


def replay(net, tree, chi, prec="f64", g=False, nets=None):
    return Emulator(describe(net, tree, chi, prec, g), nets or [net]).run()


def fwd_cases():
    out = []
    n, e = nw.square_lattice(8, 8)
    out.append(("ising 8x8 chi16", nw.ising_network(n, e, 0.44), tr.boundary_rows(8, 8), 16))
    n, e = nw.square_lattice(6, 7)
    for chi in (3, 9):
        out.append((f"normal 6x7 D3 chi{chi}", nw.random_network(n, e, 3, seed=chi), tr.boundary_rows(6, 7), chi))
    n, e = nw.square_lattice(5, 4)
    net = nw.random_network(n, e, 3, seed=2)
    out.append(("greedy 5x4 D3 chi4", net, tr.greedy(net.bonds, net.bond_dims, chi=4, seed=0), 4))
    net = nw.random_network(n, e, 3, seed=7, dist="uniform", lam=-0.2)
    out.append(("late 5x4 chi2", net, tr.from_pairs(net.bonds, tr.sequential_pairs(n), "late"), 2))
    n, e = nw.cubic_lattice(2, 2, 3)
    net = nw.ising_network(n, e, 0.5, nw.spin_glass_couplings(len(e), seed=0))
    out.append(("spin glass 2x2x3 chi2", net, tr.greedy(net.bonds, net.bond_dims, chi=2, seed=1), 2))
    net = nw.cdl_network(4, 4, 2)
    out.append(("cdl 4x4 d2 chi4", net, tr.boundary_rows(4, 4), 4))
    return out


FWD = fwd_cases()


@pytest.mark.parametrize("prec", ["f64", "tf32x3"])
@pytest.mark.parametrize("name,net,tree,chi", FWD, ids=[c[0] for c in FWD])
def test_schedule_replay_matches_oracle(name, net, tree, chi, prec):
    want = approx.contract(net, tree, chi)
    em = replay(net, tree, chi, prec)
    assert em.sign[0] == want.sign
    assert abs(em.logabs[0] - want.logabs) <= TOL * abs(want.logabs), (name, prec, em.logabs[0], want.logabs)


def test_batched_schedule_replay():
    n, e = nw.square_lattice(5, 6)
    tree = tr.boundary_rows(5, 6)
    nets = [nw.random_network(n, e, 3, seed=20 + s) for s in range(3)]
    em = replay(nets[0], tree, 5, nets=nets)
    for b, x in enumerate(nets):
        want = approx.contract(x, tree, 5)
        assert em.sign[b] == want.sign and abs(em.logabs[b] - want.logabs) <= TOL * abs(want.logabs)


def test_zero_partition_function_replay():
    edges = [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4)]
    net = nw.dimer_network(5, edges)
    em = replay(net, tr.greedy(net.bonds, net.bond_dims, chi=8), 8)
    assert em.sign[0] == 0 and em.logabs[0] == -math.inf


def grad_cases():
    out = []
    n, e = nw.square_lattice(4, 4)
    out.append(("ising 4x4 chi2", nw.ising_network(n, e, 0.44), tr.boundary_rows(4, 4), 2))
    n, e = nw.square_lattice(5, 4)
    net = nw.random_network(n, e, 3, seed=2)
    out.append(("greedy 5x4 D3 chi4", net, tr.greedy(net.bonds, net.bond_dims, chi=4, seed=0), 4))
    n, e = nw.cubic_lattice(2, 2, 3)
    net = nw.ising_network(n, e, 0.5, nw.spin_glass_couplings(len(e), seed=0))
    out.append(("spin glass 2x2x3 chi2", net, tr.greedy(net.bonds, net.bond_dims, chi=2, seed=1), 2))
    n, e = nw.square_lattice(5, 4)
    net = nw.random_network(n, e, 3, seed=7, dist="uniform", lam=-0.2)
    out.append(("late 5x4 chi2", net, tr.from_pairs(net.bonds, tr.sequential_pairs(n), "late"), 2))
    n, e = nw.square_lattice(6, 6)
    out.append(("normal 6x6 D3 chi5", nw.random_network(n, e, 3, seed=3), tr.boundary_rows(6, 6), 5))
    return out


GRAD = grad_cases()


def max_rel(ga, gb):
    scale = max(float(np.max(np.abs(x))) for x in gb)
    return max(float(np.max(np.abs(a - b))) for a, b in zip(ga, gb)) / scale


@pytest.mark.parametrize("name,net,tree,chi", GRAD, ids=[c[0] for c in GRAD])
def test_reverse_schedule_replay_matches_oracle_gradient(name, net, tree, chi):
    want = grad.contract_with_grad(net, tree, chi)
    assert want.min_gap > 1e-3 and want.min_kept > 1e-6
    em = replay(net, tree, chi, g=True)
    assert abs(em.logabs[0] - want.logabs) <= TOL * abs(want.logabs)
    got = em.grads(0, [np.shape(d) for d in net.data])
    assert max_rel(got, want.grads) <= GRAD_TOL, name


def test_reverse_schedule_mixed_form_and_batch():
    """The reverse schedule of a mixed form (tensor-core GEMM steps, emulated in FP64), batched."""
    n, e = nw.square_lattice(6, 6)
    tree = tr.boundary_rows(6, 6)
    nets = [nw.random_network(n, e, 3, seed=3), nw.random_network(n, e, 3, seed=4)]
    em = replay(nets[0], tree, 5, "tf32", g=True, nets=nets)
    for b, x in enumerate(nets):
        want = grad.contract_with_grad(x, tree, 5)
        got = em.grads(b, [np.shape(d) for d in x.data])
        if want.min_gap > 1e-3 and want.min_kept > 1e-6:
            assert max_rel(got, want.grads) <= GRAD_TOL
        for t, gv in zip(x.data, got):     # Euler's identity holds at any chi
            assert abs(float(np.sum(t * gv)) - 1.0) < 1e-9


# ---------------------------------------------------------------------------
# planted mistakes in an exported schedule must break the replay


def _mutate(plan, kind):
    p = copy.deepcopy(plan)
    steps = p["steps"]
    if kind == "transposed_operand":
        # a GEMM with a square, non-symmetric A operand reads it transposed (swapped strides)
        for st in steps:
            if st["kind"] == ST_GEMM and st["m"] == st["k"] and st["m"] > 2 and st["A"][2] != st["A"][3]:
                st["A"][2], st["A"][3] = st["A"][3], st["A"][2]
                break
        else:
            raise AssertionError("no square GEMM operand to plant the mistake in")
    elif kind == "wrong_slot":
        # a reverse rescale reads another op's exponent
        ks = [st for st in steps if st["kind"] == ST_SCALE_POW2]
        a, b = ks[0], ks[len(ks) // 2]
        a["slot"], b["slot"] = b["slot"], a["slot"]
    elif kind == "no_core_adjoint":
        p["steps"] = [st for st in steps if st["kind"] != ST_SVD_ADJ_CORE]
    return p


@pytest.mark.parametrize("kind", ["transposed_operand", "wrong_slot", "no_core_adjoint"])
def test_planted_schedule_mistakes_are_caught(kind):
    n, e = nw.square_lattice(5, 5)
    net = nw.random_network(n, e, 3, seed=11)
    tree = tr.boundary_rows(5, 5)
    plan = describe(net, tree, 4, g=True)
    good = Emulator(plan, [net]).run()
    bad = Emulator(_mutate(plan, kind), [net]).run()
    want = grad.contract_with_grad(net, tree, 4)
    gg = good.grads(0, [np.shape(d) for d in net.data])
    gb = bad.grads(0, [np.shape(d) for d in net.data])
    ok_good = abs(good.logabs[0] - want.logabs) <= TOL * abs(want.logabs) and max_rel(gg, want.grads) < 1e-6
    ok_bad = (abs(bad.logabs[0] - want.logabs) <= TOL * abs(want.logabs)
              and np.all(np.isfinite(np.concatenate([x.ravel() for x in gb]))) and max_rel(gb, want.grads) < 1e-6)
    assert ok_good and not ok_bad


def test_schedule_replay_at_the_benchmark_compression_shapes():
    """16x16, D = 4, Normal(0.2,1), chi = 64: the QR of 1024 x 256 sides and 256 x 256
    cores of the benchmark workload, through the planner's layouts."""
    n, e = nw.square_lattice(16, 16)
    net = nw.random_network(n, e, 4, seed=0)
    tree = tr.boundary_rows(16, 16)
    want = approx.contract(net, tree, 64)
    assert min(d[2] for d in want.diag) > 1e-8
    em = replay(net, tree, 64)
    assert em.sign[0] == want.sign
    assert abs(em.logabs[0] - want.logabs) <= TOL * abs(want.logabs), (em.logabs[0], want.logabs)


# ---------------------------------------------------------------------------
# checkpointed reverse pass: same gradient as one tape, less memory


@pytest.mark.parametrize("segments", [2, 3, 7, 1000])
def test_checkpointed_reverse_schedule_equals_one_tape(segments):
    n, e = nw.square_lattice(6, 6)
    net = nw.random_network(n, e, 3, seed=3)
    tree = tr.boundary_rows(6, 6)
    shapes = [np.shape(d) for d in net.data]
    full = Emulator(describe(net, tree, 5, g=True), [net]).run()
    plan = describe(net, tree, 5, g=segments)
    assert plan["segments"] == min(segments, len(tree.ops))
    ck = Emulator(plan, [net]).run()
    assert ck.logabs[0] == full.logabs[0]
    for a, b in zip(ck.grads(0, shapes), full.grads(0, shapes)):
        assert np.array_equal(a, b)      # the recomputation repeats the same steps on the same data
    want = grad.contract_with_grad(net, tree, 5)
    assert max_rel(ck.grads(0, shapes), want.grads) <= GRAD_TOL


def test_checkpointing_cuts_the_tape():
    n, e = nw.square_lattice(16, 16)
    net = nw.random_network(n, e, 4, seed=0)
    tree = tr.boundary_rows(16, 16)
    one = describe(net, tree, 64, g=True)["arena_units"]
    many = describe(net, tree, 64, g=16)["arena_units"]
    fwd = describe(net, tree, 64)["arena_units"]
    assert many < 0.25 * one and many > fwd


# ---------------------------------------------------------------------------
# tree gauge (projector form): the planned schedule against oracle.gauge


def gauge_cases():
    out = []
    n, e = nw.square_lattice(8, 8)
    out.append(("ising 8x8 chi4", nw.ising_network(n, e, 0.44), tr.boundary_rows(8, 8), 4))
    n, e = nw.square_lattice(6, 7)
    out.append(("urand 6x7 chi3", nw.random_network(n, e, 3, seed=4, dist="uniform", lam=0.0),
                tr.boundary_rows(6, 7), 3))
    net = nw.random_network(n, e, 3, seed=7)
    out.append(("normal 6x7 greedy chi5", net, tr.greedy(net.bonds, net.bond_dims, chi=5, seed=0), 5))
    return out


GAUGE = gauge_cases()


@pytest.mark.parametrize("r", [0, 1, 2, 4])
@pytest.mark.parametrize("name,net,tree,chi", GAUGE, ids=[c[0] for c in GAUGE])
def test_tree_gauge_schedule_replay_matches_oracle(name, net, tree, chi, r):
    from oracle import gauge
    want = gauge.contract_gauged(net, tree, chi, r)
    assert want.compressions > 0 and min(d[2] for d in want.diag) > 1e-8
    assert getattr(want, "min_kept", 1.0) > 1e-6, "kept values near zero: the projector form is ill-conditioned"
    from paper_2206_07044_gb300 import tn
    em = Emulator(tn.plan_describe(net, tree, chi, "f64", False, r), [net]).run()
    assert em.sign[0] == want.sign
    assert abs(em.logabs[0] - want.logabs) <= TOL * abs(want.logabs), (name, r, em.logabs[0], want.logabs)


def test_beta_sweep_configuration_plans_within_one_gpu():
    """64x64 Ising, chi = 128, TF32 form: the 256-instance beta sweep fits in HBM
    (about 0.07 GB of arena per instance; with the gradient in 64 segments about 3 GB)."""
    n, e = nw.square_lattice(64, 64)
    net = nw.ising_network(n, e, 0.44)
    tree = tr.boundary_rows(64, 64)
    p = describe(net, tree, 128, "tf32")
    assert p["arena_units"] * 8 * 256 < 64e9
    assert max(st["n"] for st in p["steps"] if st["kind"] == 3) == 256
    pg = describe(net, tree, 128, "tf32", g=64)
    assert pg["arena_units"] * 8 < 8e9
