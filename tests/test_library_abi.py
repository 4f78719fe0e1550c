"""The C-ABI library builds, loads and exports every symbol the public
header declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import subprocess

import pytest

from paper_2603_27151_gb300 import native as N


@pytest.fixture(scope="module")
def lib():
    from paper_2603_27151_gb300 import build as B
    try:
        B.build()
    except RuntimeError as e:   # no nvcc on this machine
        pytest.skip(str(e))
    return N.load()


def test_header_declares_the_boundary():
    syms = N.declared_symbols()
    for name in ("ds_soup_upload", "ds_raster_forward", "ds_raster_backward", "ds_create", "ds_destroy",
                 "ds_last_error", "ds_fragment_count", "ds_ctx_status", "ds_version", "ds_soup_free"):
        assert name in syms, name


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in N.declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    # nothing else leaks from the C++ implementation
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted({l.split()[-1] for l in out.splitlines() if " T " in l})
    assert set(exported) <= set(N.declared_symbols()) | {"_init", "_fini"}, exported


def test_version_and_error_calls_need_no_device(lib):
    assert lib.ds_version() >= 100
    assert isinstance(lib.ds_last_error(), bytes)


def test_struct_layouts_match_the_header():
    assert ctypes.sizeof(N.ds_camera) == 4 * 2 + 4 * 4 + 36 + 12 + 4
    assert ctypes.sizeof(N.ds_view_out) == 24 and ctypes.sizeof(N.ds_view_gin) == 16


def test_every_package_module_imports():
    """Each Python module of the package (and bench.py) compiles and imports
    without a GPU; the CUDA library itself is loaded only on first use."""
    import importlib
    import pkgutil
    import py_compile
    import paper_2603_27151_gb300 as pkg
    for m in pkgutil.iter_modules(pkg.__path__):
        importlib.import_module("paper_2603_27151_gb300." + m.name)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for f in ("bench.py", "__graft_entry__.py"):
        py_compile.compile(os.path.join(root, f), doraise=True)
