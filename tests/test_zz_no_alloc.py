"""tn_contract_approx_noalloc: the contraction entry point that allocates no device memory.

Callers that cannot call cudaMalloc (a plug-in whose host application's
allocator already owns the device memory, or a latency-critical path where
cudaMalloc / cudaFree would synchronise the device) use this entry point; it
draws every buffer from the library's fixed 8 MiB static device array.  Its
results must equal tn_contract_approx's on the same instance, call after call
(the array keeps the previous call's contents, so a second call checks that
everything that must start from zero is cleared).  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from tn_inputs import networks as nw
from tn_inputs import trees as tr

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _descs(net, tree):
    from paper_2206_07044_gb300.tn import NetworkDesc, TreeDesc
    dims = np.ascontiguousarray(net.bond_dims, dtype=np.int64)
    ndims = np.array([len(b) for b in net.bonds], dtype=np.int32)
    ids = np.ascontiguousarray(np.concatenate([np.asarray(b, dtype=np.int32) for b in net.bonds]), dtype=np.int32)
    arrays = [np.ascontiguousarray(d, dtype=np.float64) for d in net.data]
    ptrs = (C.POINTER(C.c_double) * len(arrays))(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrays])
    nd = NetworkDesc(len(dims), dims.ctypes.data_as(C.POINTER(C.c_int64)), len(arrays),
                     ndims.ctypes.data_as(C.POINTER(C.c_int32)), ids.ctypes.data_as(C.POINTER(C.c_int32)), ptrs)
    ops = np.ascontiguousarray(tree.as_int_array(), dtype=np.int32)
    td = TreeDesc(int(tree.n_inputs), int(ops.shape[0]), ops.ctypes.data_as(C.POINTER(C.c_int32)))
    keep = (dims, ndims, ids, arrays, ptrs, ops)
    return nd, td, keep


def _noalloc(L, net, tree, chi, stream=None):
    nd, td, keep = _descs(net, tree)
    lz = C.c_double()
    sg = C.c_int()
    msg = C.create_string_buffer(512)
    rc = L.tn_contract_approx_noalloc(C.byref(nd), C.byref(td), int(chi), C.c_void_p(stream or 0),
                                      C.byref(lz), C.byref(sg), msg, 512)
    return rc, lz.value, sg.value, msg.value.decode()


@pytest.fixture(scope="module")
def lib_and_ctx():
    import torch
    from paper_2206_07044_gb300 import build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    torch.cuda.init()
    from paper_2206_07044_gb300 import Context, tn
    L = tn.lib()
    ctx = Context(0)
    yield L, ctx
    ctx.close()


CASES = [
    ("ising 8x8 beta=0.44 chi=16", lambda: (nw.ising_network(*nw.square_lattice(8, 8), 0.44), tr.boundary_rows(8, 8), 16)),
    ("normal 6x7 D=3 chi=5", lambda: (nw.random_network(*nw.square_lattice(6, 7), 3, seed=5), tr.boundary_rows(6, 7), 5)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_noalloc_matches_allocating_entry_point_twice(lib_and_ctx, name, make):
    import torch
    L, ctx = lib_and_ctx
    net, tree, chi = make()
    want, want_sign = ctx.contract([ctx.load_tree(ctx.load_network(net), tree)], chi)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        rc, lz, sg, msg = _noalloc(L, net, tree, chi, stream)
        assert rc == 0, msg
        assert sg == int(want_sign[0])
        assert abs(lz - want[0]) <= TOL * abs(want[0]), (name, lz, want[0])


def test_noalloc_rejects_instances_beyond_its_static_scratch(lib_and_ctx):
    L, _ = lib_and_ctx
    n, edges = nw.square_lattice(16, 16)
    net = nw.random_network(n, edges, 4, seed=0)
    rc, _, _, msg = _noalloc(L, net, tr.boundary_rows(16, 16), 64)
    assert rc == -4 and "static scratch" in msg and str(8 << 20) in msg
