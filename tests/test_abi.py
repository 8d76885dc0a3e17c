"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/emt.h declares (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "emt.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(emt_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ["emt_create", "emt_destroy", "emt_load_materials", "emt_load_geometry", "emt_submit",
              "emt_run", "emt_poll", "emt_read_event", "emt_read_all"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2203_09467_gb300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    for n in declared():
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (emt_\w+)", out))
    assert set(declared()) <= exported


def test_binding_covers_every_symbol():
    from paper_2203_09467_gb300 import emt
    assert set(declared()) == set(emt._SIGS)


def test_pool_size_and_options_without_gpu():
    from paper_2203_09467_gb300 import emt
    L = emt.lib()
    o = emt.Options()
    L.emt_default_options(ctypes.byref(o))
    assert o.slot_capacity == 1 << 22 and o.max_events == 10000 and o.seed == 1
    n1 = L.emt_pool_bytes(ctypes.byref(o))
    o.slot_capacity = 1 << 23
    n2 = L.emt_pool_bytes(ctypes.byref(o))
    # two ping-pong buffers of 76 bytes per FP64 track slot
    assert n2 - n1 >= 2 * 76 * (1 << 22)
    o.precision = 1
    n3 = L.emt_pool_bytes(ctypes.byref(o))
    assert n2 - n3 >= 2 * 16 * (1 << 23)
    o.block_size = 96
    assert L.emt_pool_bytes(ctypes.byref(o)) == 0  # invalid options


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the CUDA library the binding raises."""
    import pytest
    from paper_2203_09467_gb300 import build, emt
    monkeypatch.setattr(emt, "_lib", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        emt.lib(build_if_missing=False)


def test_create_without_a_gpu_returns_the_cuda_status():
    """Without a usable GPU emt_create reports EMT_ERR_CUDA and hands out no
    context (nothing runs on the host instead)."""
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2203_09467_gb300 import emt
    L = emt.lib()
    o = emt.Options()
    L.emt_default_options(ctypes.byref(o))
    h = ctypes.c_void_p()
    assert L.emt_create(ctypes.byref(o), ctypes.byref(h)) == -3
    assert h.value is None
