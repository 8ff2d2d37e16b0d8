"""The C-ABI library builds, loads and exports every symbol include/tn.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "tn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2206_07044_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for need in ("tn_create", "tn_destroy", "tn_load_network", "tn_load_tree", "tn_contract_approx",
                 "tn_last_error", "tn_set_stream"):
        assert need in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2206_07044_gb300 import tn
    assert set(declared_symbols()) <= set(tn.SIGNATURES)


def test_version_and_null_handling(libpath):
    from paper_2206_07044_gb300 import tn
    L = tn.lib()
    assert L.tn_version().decode().startswith("tn-gb300")
    assert L.tn_last_error(None) == b"NULL context"
    assert L.tn_create(None, 0, None) == -1     # TN_EINVAL on a NULL out-pointer
    opt = tn.Options()
    L.tn_options_default(ctypes.byref(opt))
    assert opt.struct_size == ctypes.sizeof(tn.Options) and opt.graph_mode == 1
    assert opt.grad_segments == 0 and opt.debug_max_sweeps == 0 and opt.tape_budget_bytes == 0.0
    h = ctypes.c_void_p()
    bad = tn.Options()
    L.tn_options_default(ctypes.byref(bad))
    bad.struct_size = 4                         # an options struct older than the first version
    assert L.tn_create(ctypes.byref(h), 0, ctypes.byref(bad)) == -1
    L.tn_options_default(ctypes.byref(bad))
    bad.debug_max_sweeps = -1
    assert L.tn_create(ctypes.byref(h), 0, ctypes.byref(bad)) == -1
    L.tn_destroy(None)                          # ignored


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2206_07044_gb300 import tn
    with pytest.raises(tn.TNError):
        tn.Context(0)


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    from paper_2206_07044_gb300 import tn
    monkeypatch.setattr(tn, "_LIB", None)
    monkeypatch.setattr(tn, "LIB_PATH", str(tmp_path / "libtn.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        tn.lib()
