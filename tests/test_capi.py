"""The C-ABI library loads and exports every entry point declared in include/vga.h; host-side
argument validation answers before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vga():
    from paper_2406_04177_gb300 import build

    build.build()
    import paper_2406_04177_gb300 as v

    v.load_library()
    return v


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(vga_[a-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    assert "vga_graph_build" in names and "vga_sim_step" in names and len(names) >= 20


def test_every_declared_symbol_is_exported(vga):
    lib = vga.load_library()
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in include/*.h but not exported by libvga.so"


def test_binding_covers_every_declared_symbol(vga):
    assert sorted(vga.declared_symbols()) == _declared()
    for name in _declared():
        assert callable(getattr(vga, name)), name


def test_strerror_and_version(vga):
    assert vga.vga_strerror(0) == "VGA_OK"
    for code, name in vga.STATUS_NAMES.items():
        assert vga.vga_strerror(code) == name
    assert vga.vga_strerror(-99) == "VGA_ERR_UNKNOWN"
    assert vga.vga_version() >= 10000


def test_graph_build_rejects_bad_sizes_without_device_work(vga):
    lib = vga.load_library()
    out = C.c_void_p()
    img = np.zeros(8, dtype=np.uint8)
    p = img.ctypes.data_as(C.c_void_p)
    for dims in [(0, 2, 2), (2, -1, 2), (40000, 1, 1), (2048, 2048, 1024)]:
        assert lib.vga_graph_build(p, *dims, 1, None, C.byref(out)) == -1
        assert out.value is None
    assert lib.vga_graph_build(None, 2, 2, 2, 1, None, C.byref(out)) == -1
    assert lib.vga_graph_build(p, 2, 2, 2, 1 << 7, None, C.byref(out)) == -1
    assert "flags" in vga.vga_last_error()
    assert lib.vga_graph_build(p, 2, 2, 2, 1, None, None) == -1


def test_sim_calls_reject_null_handles(vga):
    lib = vga.load_library()
    out = C.c_void_p()
    pp = vga.make_params(dict(D=1, dt=0.1, rho=0, mu=0, beta=0.5, v_som=0, v_fom=0, v_dom=0, K_dom=1))
    assert lib.vga_sim_create(None, C.byref(pp), None, C.byref(out)) == -1
    assert lib.vga_sim_step(None, 1) == -1
    assert lib.vga_sim_totals(None, None) == -1
    assert lib.vga_graph_info(None, None, None, None) == -1
    assert lib.vga_graph_free(None) == 0 and lib.vga_sim_free(None) == 0


def test_no_cpu_fallback_when_library_missing(tmp_path):
    """The binding raises instead of computing anything when the library is absent."""
    import importlib

    import paper_2406_04177_gb300 as v

    mod = importlib.reload(v)
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            mod.load_library(str(tmp_path / "missing.so"))
    finally:
        importlib.reload(v)


def test_noalloc_wrapper_rejects_short_or_strided_buffers():
    """The Python wrapper of the allocation-free totals checks sizes and layout before any device
    access (the kernel has no bounds of its own to check); no GPU is needed to see the rejections."""
    import torch

    import paper_2406_04177_gb300 as v

    n, stride = 100, 120
    ok_vals = torch.zeros(4 * stride + n, dtype=torch.float32)
    ok_tot = torch.zeros(5, dtype=torch.float64)
    with pytest.raises(ValueError, match="values holds"):
        v.vga_state_totals_noalloc(torch.zeros(4 * stride + n - 1), None, n, stride, ok_tot)
    with pytest.raises(ValueError, match="residuals holds"):
        v.vga_state_totals_noalloc(ok_vals, torch.zeros(4 * stride, dtype=torch.int16), n, stride, ok_tot)
    with pytest.raises(ValueError, match="totals holds"):
        v.vga_state_totals_noalloc(ok_vals, None, n, stride, torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError, match="contiguous"):
        v.vga_state_totals_noalloc(torch.zeros(2 * (4 * stride + n))[::2], None, n, stride, ok_tot)
    with pytest.raises(ValueError, match="row_stride"):
        v.vga_state_totals_noalloc(ok_vals, None, n, n - 1, ok_tot)
    with pytest.raises(ValueError, match="row_stride"):
        v.vga_state_totals_noalloc(ok_vals, None, -1, stride, ok_tot)
    # sizes right, but host tensors: refused before the library is called
    with pytest.raises(TypeError, match="CUDA"):
        v.vga_state_totals_noalloc(ok_vals, None, n, stride, ok_tot)
