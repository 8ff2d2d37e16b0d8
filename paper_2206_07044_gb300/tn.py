"""Thin ctypes binding of ``libtn.so`` (include/tn.h): argument marshalling only.

Every step of the contraction runs in the library's CUDA kernels; this module
converts Python objects to plain pointers and sizes and raises
:class:`TNError` on any non-OK status.  It never computes a result itself and
has no CPU fallback: if ``libtn.so`` is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtn.so")

TN_F64, TN_TF32, TN_BF16, TN_TF32X3 = 0, 1, 2, 3
PREC = {"f64": TN_F64, "tf32": TN_TF32, "bf16": TN_BF16, "tf32x3": TN_TF32X3}

STATUS = {0: "TN_OK", -1: "TN_EINVAL", -2: "TN_EFORMAT", -3: "TN_ESHAPE", -4: "TN_ENOMEM",
          -5: "TN_ECUDA", -6: "TN_ETIMEOUT", -7: "TN_ENONFINITE", -8: "TN_ESTATE", -9: "TN_ENOCONV"}


class TNError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class NetworkDesc(C.Structure):
    _fields_ = [("n_bonds", C.c_int32), ("bond_dims", C.POINTER(C.c_int64)),
                ("n_tensors", C.c_int32), ("ndims", C.POINTER(C.c_int32)),
                ("bond_ids", C.POINTER(C.c_int32)), ("data", C.POINTER(C.POINTER(C.c_double)))]


class TreeDesc(C.Structure):
    _fields_ = [("n_inputs", C.c_int32), ("n_ops", C.c_int32), ("ops", C.POINTER(C.c_int32))]


class PlanStats(C.Structure):
    _fields_ = [("n_contractions", C.c_int64), ("n_compressions", C.c_int64),
                ("gemm_flops", C.c_double), ("qr_flops", C.c_double), ("svd_flops", C.c_double),
                ("permute_bytes", C.c_double), ("peak_bytes", C.c_double),
                ("kernel_launches", C.c_int64)]


class Options(C.Structure):
    _fields_ = [("struct_size", C.c_int32), ("graph_mode", C.c_int32), ("grad_segments", C.c_int32),
                ("debug_max_sweeps", C.c_int32), ("tape_budget_bytes", C.c_double),
                ("debug_tc_give_up", C.c_int32), ("reserved", C.c_int32), ("tuner_cache", C.c_char_p),
                ("sequential_groups", C.c_int32), ("split_batches", C.c_int32)]


# every symbol include/tn.h declares, with its ctypes signature
SIGNATURES = {
    "tn_version": (C.c_char_p, []),
    "tn_options_default": (None, [C.POINTER(Options)]),
    "tn_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(Options)]),
    "tn_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "tn_tuned_choices": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int32)]),
    "tn_destroy": (None, [C.c_void_p]),
    "tn_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tn_set_graph_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "tn_graph_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "tn_load_network": (C.c_int, [C.c_void_p, C.POINTER(NetworkDesc), C.POINTER(C.c_int)]),
    "tn_load_network_file": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_int)]),
    "tn_set_network_data": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.c_int]),
    "tn_load_tree": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(TreeDesc), C.POINTER(C.c_int)]),
    "tn_load_tree_file": (C.c_int, [C.c_void_p, C.c_int, C.c_char_p, C.POINTER(C.c_int)]),
    "tn_contract_approx": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int,
                                     C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "tn_grad": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(C.c_double),
                          C.POINTER(C.c_int), C.POINTER(C.c_void_p), C.c_int]),
    "tn_set_grad_segments": (C.c_int, [C.c_void_p, C.c_int]),
    "tn_plan_describe": (C.c_int, [C.POINTER(NetworkDesc), C.POINTER(TreeDesc), C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "tn_set_tree_gauge": (C.c_int, [C.c_void_p, C.c_int]),
    "tn_plan_stats_get": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(PlanStats)]),
    "tn_debug_tensor": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.c_int, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "tn_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "tn_kernel_times": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_char_p),
                                  C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "tn_last_error": (C.c_char_p, [C.c_void_p]),
    "tn_contract_approx_noalloc": (C.c_int, [C.POINTER(NetworkDesc), C.POINTER(TreeDesc), C.c_int, C.c_void_p,
                                             C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_char_p, C.c_size_t]),
}

_LIB: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    """Load libtn.so (built by ``paper_2206_07044_gb300.build``); raise if absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2206_07044_gb300.build.build() first "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def plan_describe(net, tree, chi: int, prec="f64", grad=False, gauge_r: int = -1) -> dict:
    """The library's static schedule for (network structure, tree, chi, form) as a dict.

    grad: False (forward), True (with the reverse pass) or k >= 2 (reverse pass
    checkpointed in k segments).

    Needs no context and no GPU (host planning only); see tn_plan_describe in
    include/tn.h for the fields.
    """
    import json
    L = lib()
    dims = np.ascontiguousarray(net.bond_dims, dtype=np.int64)
    ndims = np.array([len(b) for b in net.bonds], dtype=np.int32)
    ids = np.ascontiguousarray(np.concatenate([np.asarray(b, dtype=np.int32) for b in net.bonds])
                               if sum(ndims) else np.zeros(1, np.int32), dtype=np.int32)
    desc = NetworkDesc(len(dims), dims.ctypes.data_as(C.POINTER(C.c_int64)), len(net.bonds),
                       ndims.ctypes.data_as(C.POINTER(C.c_int32)), ids.ctypes.data_as(C.POINTER(C.c_int32)), None)
    ops = np.ascontiguousarray(tree.as_int_array(), dtype=np.int32)
    if ops.size == 0:
        ops = np.zeros((0, 4), np.int32)
    tdesc = TreeDesc(int(tree.n_inputs), int(ops.shape[0]), ops.ctypes.data_as(C.POINTER(C.c_int32)) if ops.size else None)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    need = C.c_size_t()
    g = int(grad) if not isinstance(grad, bool) else (1 if grad else 0)
    rc = L.tn_plan_describe(C.byref(desc), C.byref(tdesc), int(chi), p, g, int(gauge_r), None, 0, C.byref(need))
    if rc != 0:
        raise TNError(rc, "tn_plan_describe failed")
    buf = C.create_string_buffer(need.value)
    rc = L.tn_plan_describe(C.byref(desc), C.byref(tdesc), int(chi), p, g, int(gauge_r), buf, need.value,
                            C.byref(need))
    if rc != 0:
        raise TNError(rc, "tn_plan_describe failed")
    return json.loads(buf.value.decode())


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, stream=None, **options):
        """options: any field of tn_options (graph_mode, grad_segments,
        tape_budget_bytes, debug_max_sweeps, debug_tc_give_up, tuner_cache,
        sequential_groups, split_batches); the rest keep their defaults."""
        self._L = lib()
        opt = Options()
        self._L.tn_options_default(C.byref(opt))
        for k, v in options.items():
            if k in ("struct_size", "reserved") or k not in dict(Options._fields_):
                raise TypeError(f"unknown tn_options field {k!r}")
            if k == "tuner_cache":
                self._tuner_cache = v.encode() if isinstance(v, str) else v
                v = self._tuner_cache
            setattr(opt, k, v)
        h = C.c_void_p()
        rc = self._L.tn_create(C.byref(h), int(device), C.byref(opt))
        if rc != 0:
            raise TNError(rc, f"tn_create(device={device}) failed (no CUDA device?)")
        self._h = h
        self.device = device
        self._shapes: Dict[int, List[Tuple[int, ...]]] = {}   # net id -> tensor shapes
        self._inst_net: Dict[int, int] = {}                   # instance id -> net id
        if stream is not None:
            self.set_stream(stream)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._L.tn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int) -> None:
        if rc != 0:
            raise TNError(rc, self._L.tn_last_error(self._h).decode())

    def set_stream(self, stream) -> None:
        self._check(self._L.tn_set_stream(self._h, C.c_void_p(_stream_handle(stream))))

    def load_network(self, net) -> int:
        """net: an object with bond_dims, bonds (per tensor) and data (float64 arrays)."""
        dims = np.ascontiguousarray(net.bond_dims, dtype=np.int64)
        ndims = np.array([len(b) for b in net.bonds], dtype=np.int32)
        ids = np.ascontiguousarray(np.concatenate([np.asarray(b, dtype=np.int32) for b in net.bonds])
                                   if sum(ndims) else np.zeros(1, np.int32), dtype=np.int32)
        arrays = [np.ascontiguousarray(d, dtype=np.float64) for d in net.data]
        ptrs = (C.POINTER(C.c_double) * len(arrays))(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrays])
        desc = NetworkDesc(len(dims), dims.ctypes.data_as(C.POINTER(C.c_int64)), len(arrays),
                           ndims.ctypes.data_as(C.POINTER(C.c_int32)), ids.ctypes.data_as(C.POINTER(C.c_int32)),
                           ptrs)
        out = C.c_int()
        self._check(self._L.tn_load_network(self._h, C.byref(desc), C.byref(out)))
        self._shapes[out.value] = [tuple(int(net.bond_dims[b]) for b in bl) for bl in net.bonds]
        return out.value

    def load_network_file(self, path: str) -> int:
        out = C.c_int()
        self._check(self._L.tn_load_network_file(self._h, path.encode(), C.byref(out)))
        return out.value

    def set_network_data(self, net_id: int, tensors: Sequence, on_device: bool = False) -> None:
        """Replace a network's entries: host float64 arrays, or device pointers / CUDA tensors."""
        keep = []
        ptrs = []
        for t in tensors:
            if on_device:
                ptrs.append(int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t))
            elif hasattr(t, "data_ptr"):
                # a host torch tensor (e.g. pinned): its storage is passed as is
                if not (t.is_contiguous() and str(t.dtype) == "torch.float64" and t.device.type == "cpu"):
                    raise ValueError("host tensors must be contiguous float64 CPU tensors")
                keep.append(t)
                ptrs.append(int(t.data_ptr()))
            else:
                a = np.ascontiguousarray(t, dtype=np.float64)
                keep.append(a)
                ptrs.append(a.ctypes.data)
        arr = (C.c_void_p * len(ptrs))(*ptrs)
        self._check(self._L.tn_set_network_data(self._h, int(net_id), arr, 1 if on_device else 0))
        self._keep_alive = keep

    def load_tree(self, net_id: int, tree) -> int:
        ops = np.ascontiguousarray(tree.as_int_array(), dtype=np.int32)
        if ops.size == 0:
            ops = np.zeros((0, 4), np.int32)
        desc = TreeDesc(int(tree.n_inputs), int(ops.shape[0]),
                        ops.ctypes.data_as(C.POINTER(C.c_int32)) if ops.size else None)
        out = C.c_int()
        self._check(self._L.tn_load_tree(self._h, int(net_id), C.byref(desc), C.byref(out)))
        self._inst_net[out.value] = int(net_id)
        return out.value

    def load_tree_file(self, net_id: int, path: str) -> int:
        out = C.c_int()
        self._check(self._L.tn_load_tree_file(self._h, int(net_id), path.encode(), C.byref(out)))
        return out.value

    def contract(self, inst_ids: Iterable[int], chi: int, prec="f64") -> Tuple[np.ndarray, np.ndarray]:
        """(log|Z|, sign) per instance, computed on the GPU."""
        ids = np.ascontiguousarray(list(inst_ids), dtype=np.int32)
        n = len(ids)
        logz = np.zeros(n, dtype=np.float64)
        sign = np.zeros(n, dtype=np.int32)
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        self._check(self._L.tn_contract_approx(self._h, n, ids.ctypes.data_as(C.POINTER(C.c_int)), int(chi), p,
                                               logz.ctypes.data_as(C.POINTER(C.c_double)),
                                               sign.ctypes.data_as(C.POINTER(C.c_int))))
        return logz, sign

    def set_tree_gauge(self, r: int) -> None:
        """Compress in the tree gauge of distance r (projector form); -1 restores the plain Q-form."""
        self._check(self._L.tn_set_tree_gauge(self._h, int(r)))

    def set_grad_segments(self, segments: int) -> None:
        """Checkpoint tn_grad's tape in `segments` segments (1: one tape; 0: by free memory)."""
        self._check(self._L.tn_set_grad_segments(self._h, int(segments)))

    def shapes(self, inst_id: int) -> List[Tuple[int, ...]]:
        """Tensor shapes of an instance's network (networks loaded from arrays)."""
        return self._shapes[self._inst_net[inst_id]]

    def grad(self, inst_ids: Sequence[int], chi: int, prec="f64", out=None):
        """(log|Z|, sign, gradients): d log|Z| / d T_v for every input tensor, on the GPU.

        Without ``out``, returns per instance a list of host arrays shaped like the
        inputs.  ``out``: one buffer per instance (numpy arrays, or CUDA tensors
        passed by device pointer) of sum_t |T_t| float64 values, filled packed.
        """
        ids = np.ascontiguousarray(list(inst_ids), dtype=np.int32)
        n = len(ids)
        logz = np.zeros(n, dtype=np.float64)
        sign = np.zeros(n, dtype=np.int32)
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        on_device = False
        if out is None:
            shapes = [self.shapes(int(i)) for i in ids]
            out = [np.zeros(sum(int(np.prod(s, dtype=np.int64)) for s in sh), dtype=np.float64) for sh in shapes]
        ptrs = []
        for o in out:
            if hasattr(o, "data_ptr"):
                on_device = o.device.type == "cuda"
                if not (o.is_contiguous() and str(o.dtype) == "torch.float64"):
                    raise ValueError("gradient buffers must be contiguous float64")
                ptrs.append(int(o.data_ptr()))
            else:
                if o.dtype != np.float64 or not o.flags["C_CONTIGUOUS"]:
                    raise ValueError("gradient buffers must be contiguous float64")
                ptrs.append(o.ctypes.data)
        arr = (C.c_void_p * n)(*ptrs)
        self._check(self._L.tn_grad(self._h, n, ids.ctypes.data_as(C.POINTER(C.c_int)), int(chi), p,
                                    logz.ctypes.data_as(C.POINTER(C.c_double)),
                                    sign.ctypes.data_as(C.POINTER(C.c_int)), arr, 1 if on_device else 0))
        if on_device or hasattr(out[0], "data_ptr"):
            return logz, sign, out
        grads = []
        for i, o in zip(ids, out):
            parts, off = [], 0
            for s in self.shapes(int(i)):
                sz = int(np.prod(s, dtype=np.int64))
                parts.append(o[off:off + sz].reshape(s))
                off += sz
            grads.append(parts)
        return logz, sign, grads

    def debug_tensor(self, inst_ids: Sequence[int], which: int, chi: int, stop_op: int, tensor_id: int,
                     prec="f64") -> Tuple[np.ndarray, List[int]]:
        """Tensor `tensor_id` of instance inst_ids[which] after tree op `stop_op` (GPU-computed).

        Returns (array shaped by its storage order, bond ids in that order).
        """
        ids = np.ascontiguousarray(list(inst_ids), dtype=np.int32)
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        nd = C.c_int32()
        bonds = (C.c_int32 * 24)()
        dims = (C.c_int64 * 24)()
        args = (self._h, len(ids), ids.ctypes.data_as(C.POINTER(C.c_int)), int(which), int(chi), p, int(stop_op),
                int(tensor_id))
        self._check(self._L.tn_debug_tensor(*args, None, 0, C.byref(nd), bonds, dims))
        shape = [int(dims[a]) for a in range(nd.value)]
        out = np.zeros(int(np.prod(shape, dtype=np.int64)), dtype=np.float64)
        self._check(self._L.tn_debug_tensor(*args, out.ctypes.data_as(C.POINTER(C.c_double)), out.size,
                                            C.byref(nd), bonds, dims))
        return out.reshape(shape), [int(bonds[a]) for a in range(nd.value)]

    def autotune(self, inst_ids: Sequence[int], chi: int, prec="f64") -> int:
        """Time the candidate launch shapes of this batch's plan and keep the fastest (tn_autotune)."""
        ids = np.ascontiguousarray(list(inst_ids), dtype=np.int32)
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        n = C.c_int()
        self._check(self._L.tn_autotune(self._h, len(ids), ids.ctypes.data_as(C.POINTER(C.c_int)), int(chi), p,
                                        C.byref(n)))
        return n.value

    def tuned_choices(self) -> List[Tuple[int, int, int, int, int, int]]:
        """The device's tuned choices: (family, m, n, k, batch, choice) rows (tn_tuned_choices)."""
        cnt = self._L.tn_tuned_choices(self._h, 0, None)
        if cnt < 0:
            self._check(cnt)
        buf = (C.c_int32 * (6 * max(cnt, 1)))()
        self._L.tn_tuned_choices(self._h, cnt, buf)
        return [tuple(int(buf[6 * i + j]) for j in range(6)) for i in range(cnt)]

    def plan_stats(self, inst_id: int, chi: int, prec="f64") -> Dict[str, float]:
        st = PlanStats()
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        self._check(self._L.tn_plan_stats_get(self._h, int(inst_id), int(chi), p, C.byref(st)))
        return {k: getattr(st, k) for k, _ in PlanStats._fields_}

    def set_graph_mode(self, enable: bool) -> None:
        """Replay whole schedules as CUDA graphs (default on) or launch every kernel eagerly."""
        self._check(self._L.tn_set_graph_mode(self._h, 1 if enable else 0))

    def graph_info(self) -> dict:
        """Graphs captured, replays launched and captures refused since the context was made."""
        v = [C.c_int64() for _ in range(3)]
        self._check(self._L.tn_graph_info(self._h, *[C.byref(x) for x in v]))
        return {"captured": v[0].value, "replays": v[1].value, "refused": v[2].value}

    def profile(self, enable: bool) -> None:
        self._check(self._L.tn_profile_enable(self._h, 1 if enable else 0))

    def kernel_times(self) -> List[Tuple[str, int, float]]:
        cap = 32
        names = (C.c_char_p * cap)()
        launches = (C.c_int64 * cap)()
        ms = (C.c_double * cap)()
        n = self._L.tn_kernel_times(self._h, cap, names, launches, ms)
        return [(names[i].decode(), int(launches[i]), float(ms[i])) for i in range(min(n, cap))]


def version() -> str:
    return lib().tn_version().decode()
