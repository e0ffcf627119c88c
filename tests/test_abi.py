"""The C-ABI library builds, loads without a GPU and exports every symbol include/gbcfd.h
declares; the Python binding wraps exactly those entry points."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gbcfd_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1710_09995_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_calls():
    names = set(declared_functions())
    for call in ("create_block", "set_metrics", "set_state", "compute_residual", "step",
                 "exchange_halos", "residual_norm"):
        assert f"gbcfd_{call}" in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_exactly_the_declared_symbols():
    from paper_1710_09995_gb300 import gbcfd
    assert set(gbcfd.SIGNATURES) == set(declared_functions())


def test_library_is_built_for_sm_103a_only(libpath):
    from paper_1710_09995_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_pipeline_argument_checks_need_no_device(libpath):
    """the pipeline entry points refuse null handles and bad counts on the host, before any CUDA
    call (so these run without a GPU)"""
    from paper_1710_09995_gb300 import gbcfd
    lib = gbcfd.lib()
    out = ctypes.c_void_p(0)
    one = (ctypes.c_void_p * 1)(None)
    assert lib.gbcfd_pipe_create(None, 1, ctypes.byref(out)) == gbcfd.ERR_ARG
    assert lib.gbcfd_pipe_create(one, 0, ctypes.byref(out)) == gbcfd.ERR_ARG
    assert lib.gbcfd_pipe_create(one, 9, ctypes.byref(out)) == gbcfd.ERR_ARG
    assert lib.gbcfd_pipe_create(one, 1, ctypes.byref(out)) == gbcfd.ERR_ARG  # a NULL block
    assert b"NULL block" in lib.gbcfd_last_error()
    assert lib.gbcfd_wcns_pipe_create(one, 1, ctypes.byref(out)) == gbcfd.ERR_ARG
    assert lib.gbcfd_group_pipe_create(one, 1, ctypes.byref(out)) == gbcfd.ERR_ARG
    assert lib.gbcfd_group_pipe_create(one, 0, ctypes.byref(out)) == gbcfd.ERR_ARG
    assert out.value is None
    assert lib.gbcfd_pipe_submit(None, None, None, 1, None) == gbcfd.ERR_ARG
    assert lib.gbcfd_pipe_sync(None) == gbcfd.ERR_ARG
    assert lib.gbcfd_pipe_destroy(None) == gbcfd.ERR_ARG


def test_header_is_plain_c():
    """include/gbcfd.h compiles as C99 (no C++ or torch types cross the boundary)"""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    r = subprocess.run([cc, "-fsyntax-only", "-std=c99", "-Wall", "-Werror", "-x", "c",
                        os.path.join(ROOT, "include", "gbcfd.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
