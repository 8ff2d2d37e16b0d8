"""Bounded device loops report their failure and leave the context usable (GPU).

Nothing here faults or hangs a GPU: each test caps a loop or a wait through a
context option, so that the kernel gives up early, records an error status
that the host reads, and returns.
"""
import pytest

from oracle import approx
from tn_inputs import networks as nw
from tn_inputs import trees as tr

pytestmark = pytest.mark.gpu


def _ctx(**opt):
    import torch
    from paper_2206_07044_gb300 import Context, build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return Context(0, **opt)


def test_jacobi_sweep_cap_returns_enoconv_and_device_stays_usable():
    """The FP64 polish of the core SVD needs 2-3 sweeps from the FP32 start; a cap of one
    sweep makes every core report non-convergence (TN_ENOCONV), and the next call on a
    context without the cap is exact again."""
    from paper_2206_07044_gb300.tn import TNError
    n, e = nw.square_lattice(8, 8)
    net = nw.ising_network(n, e, 0.44)
    tree = tr.boundary_rows(8, 8)
    capped = _ctx(debug_max_sweeps=1, graph_mode=0)
    iid = capped.load_tree(capped.load_network(net), tree)
    with pytest.raises(TNError) as ei:
        capped.contract([iid], 16)
    assert ei.value.code == -9
    # the capped context itself still runs exact contractions (no compression fires at chi = 1024)
    lz, sg = capped.contract([iid], 1024)
    capped.close()
    fresh = _ctx()
    iid2 = fresh.load_tree(fresh.load_network(net), tree)
    lz2, sg2 = fresh.contract([iid2], 16)
    fresh.close()
    want = approx.contract(net, tree, 16)
    assert sg2[0] == want.sign and abs(lz2[0] - want.logabs) <= 1e-10 * abs(want.logabs)
    exact_lz = approx.contract(net, tree, None).logabs
    assert abs(lz[0] - exact_lz) <= 1e-12 * abs(exact_lz)


def test_tensor_core_wait_give_up_returns_etimeout_and_device_stays_usable():
    """With the tensor-core GEMM's pipeline waits set to give up at once, every GEMM of a
    mixed form drains its copies, frees its TMEM and flags the call: TN_ETIMEOUT.  The same
    context then runs the FP64 form (no tensor-core GEMM) exactly, and a fresh context runs
    the mixed form again."""
    from paper_2206_07044_gb300.tn import TNError
    n, e = nw.square_lattice(6, 6)
    net = nw.random_network(n, e, 2, seed=3)
    tree = tr.boundary_rows(6, 6)
    c = _ctx(debug_tc_give_up=1, graph_mode=0)
    iid = c.load_tree(c.load_network(net), tree)
    for prec in ("tf32", "bf16", "tf32x3"):
        with pytest.raises(TNError) as ei:
            c.contract([iid], 4, prec)
        assert ei.value.code == -6, prec
    want = approx.contract(net, tree, 4)
    lz, sg = c.contract([iid], 4, "f64")
    c.close()
    assert sg[0] == want.sign and abs(lz[0] - want.logabs) <= 1e-10 * abs(want.logabs)
    fresh = _ctx()
    iid2 = fresh.load_tree(fresh.load_network(net), tree)
    lz2, _ = fresh.contract([iid2], 4, "tf32x3")
    fresh.close()
    assert abs(lz2[0] - want.logabs) <= 2.0 ** -11 * abs(want.logabs)
