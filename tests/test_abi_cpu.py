"""CPU-side checks of the boundary: the library builds, loads and exports every symbol
that include/tcm.h declares; the binding's structure layouts match the header.
No compute call is made (there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tcm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tcm_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_0704_1672_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tcm_ctx_create", "tcm_ctx_destroy", "tcm_last_error", "tcm_moments", "tcm_energy",
              "tcm_energy_batch", "tcm_direct", "tcm_prepare", "tcm_ctx_set_stream"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.tcm_last_error.restype = ctypes.c_char_p
    assert lib.tcm_last_error() == b""


def test_context_create_fails_cleanly_without_gpu(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = ctypes.CDLL(libpath)
    lib.tcm_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p(123)
    rc = lib.tcm_ctx_create(ctypes.byref(h), 10, None)
    assert rc != 0 and h.value is None
    assert len(lib.tcm_last_error()) > 0
    rc = lib.tcm_ctx_create(ctypes.byref(h), 99, None)
    assert rc == 1  # TCM_EINVAL for lmax_cap out of range


def test_struct_layouts_match_header():
    from paper_0704_1672_gb300 import tcm
    assert ctypes.sizeof(tcm.tcm_system) == 8 + 8 + 4 + 4 + 24 + 8 + 8 + 4 + 4
    assert ctypes.sizeof(tcm.tcm_moments_t) == 8 + 4 + 4 + 24 + 8
    assert ctypes.sizeof(tcm.tcm_pair_item) == 16 + 72 + 24
    assert tcm.PAIR_ITEM_DTYPE.itemsize == ctypes.sizeof(tcm.tcm_pair_item)


def test_unbuilt_library_fails_loudly(monkeypatch, tmp_path):
    from paper_0704_1672_gb300 import tcm
    monkeypatch.setattr(tcm, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(tcm, "_lib", None)
    with pytest.raises(tcm.TcmError):
        tcm.lib()
