"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
and exports every entry point that include/helmmg.h declares.  No compute
calls are made (no GPU here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "helmmg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2308_13476_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mg_setup", "mg_solve", "mg_adjoint", "mg_gradient", "mg_destroy", "mg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    import paper_2308_13476_gb300 as hm
    assert sorted(hm.EXPORTED) == declared_functions()


def test_default_options_and_error_paths_without_gpu(lib_path):
    import paper_2308_13476_gb300 as hm
    o = hm.mg_default_options()
    assert (o.cycle, o.smoother, o.nu_pre, o.nu_post, o.omega, o.precision) == (1, 0, 1, 1, 4.5, 0)
    assert (o.max_cycles, o.min_coarse, o.batch) == (10000, 10, 1)
    lib = hm.load_library()
    h = ctypes.c_void_p()
    # argument validation happens before any device call
    st = lib.mg_setup(ctypes.byref(h), 1, 8, 0.1, None, 5.0, 0.7, 0, ctypes.byref(o))
    assert st == hm.MG_EINVAL and h.value is None
    assert b"nx, ny >= 2" in lib.mg_last_error()
    assert lib.mg_destroy(None) == hm.MG_OK


def test_options_struct_matches_the_header():
    """The ctypes mirror of mg_options lists the header's fields in order."""
    import paper_2308_13476_gb300 as hm
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} mg_options;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:int|double|void\s*\*)\s*\**\s*([a-z_0-9]+)\s*;", body)
    assert fields == [f[0] for f in hm.MgOptions._fields_]


def test_krylov_option_validated_without_gpu(lib_path):
    import paper_2308_13476_gb300 as hm
    lib = hm.load_library()
    o = hm.mg_default_options()
    assert o.krylov == 0
    h = ctypes.c_void_p()
    o.krylov = 33
    assert lib.mg_setup(ctypes.byref(h), 8, 8, 0.1, None, 5.0, 0.7, 0, ctypes.byref(o)) == hm.MG_EINVAL
    assert b"krylov" in lib.mg_last_error()
    o.krylov, o.precision = 4, 2
    assert lib.mg_setup(ctypes.byref(h), 8, 8, 0.1, None, 5.0, 0.7, 0, ctypes.byref(o)) == hm.MG_EINVAL
    assert b"precision 0 or 1" in lib.mg_last_error()
    assert h.value is None


def test_transfer_option_validated_without_gpu(lib_path):
    import paper_2308_13476_gb300 as hm
    lib = hm.load_library()
    o = hm.mg_default_options()
    assert o.transfer == 0
    h = ctypes.c_void_p()
    o.transfer = 2
    assert lib.mg_setup(ctypes.byref(h), 8, 8, 0.1, None, 5.0, 0.7, 0, ctypes.byref(o)) == hm.MG_EINVAL
    assert b"transfer" in lib.mg_last_error()
    assert h.value is None


def test_two_grid_and_profile_arguments_validated_without_gpu(lib_path):
    import paper_2308_13476_gb300 as hm
    lib = hm.load_library()
    out = (ctypes.c_double * 6)()
    assert lib.mg_two_grid(None, 1, 1000, out) == hm.MG_EINVAL
    ms, nb = ctypes.c_double(), ctypes.c_double()
    assert lib.mg_profile(None, 5, 0, 1, ctypes.byref(ms), ctypes.byref(nb)) == hm.MG_EINVAL
