"""The C-ABI library loads without a GPU and exports every entry point that
include/mhd.h declares; the Python binding declares a signature for each."""
import ctypes
import os
import re

from paper_2609_10849_b300 import mhd

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mhd.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mhd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("mhd_create", "mhd_set_params", "mhd_set_stream", "mhd_set_state", "mhd_get_state",
                 "mhd_set_B_from_potential", "mhd_compute_dt", "mhd_strang_step", "mhd_substep",
                 "mhd_adjoint_step", "mhd_diagnostics", "mhd_batch_create", "mhd_batch_step", "mhd_destroy",
                 "mhd_status_string", "mhd_last_error"):
        assert must in names, must


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(mhd.LIB_PATH)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    missing = [n for n in declared() if n not in mhd._SIGS]
    assert not missing, missing


def test_debug_library_exports_the_same_symbols():
    """The index-checking build exports the same entry points (and says so)."""
    path = os.path.join(os.path.dirname(mhd.LIB_PATH), "libmhd_debug.so")
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    rel = ctypes.CDLL(os.path.join(os.path.dirname(mhd.LIB_PATH), "libmhd.so"))
    rel.mhd_debug_oob.restype = ctypes.c_longlong
    assert rel.mhd_debug_oob(0) == -1  # the release build has no checks
