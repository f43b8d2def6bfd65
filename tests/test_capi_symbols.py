"""The C-ABI library builds, loads and exports every function include/pabd.h declares
(CPU only: no function that touches the device is called)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"^\s*(?:pabd_status|const char\*)\s+(pabd_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    return ctypes.CDLL(os.path.join(ROOT, "paper_2609_02675_gb300", "libpabd.so"))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"pabd_create_scene", "pabd_add_body", "pabd_add_bond", "pabd_step", "pabd_read_state"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_the_abi(lib):
    import paper_2609_02675_gb300 as P
    assert set(P.EXPORTED) == _declared()
    for n in P.EXPORTED:
        if n not in ("pabd_status_str", "pabd_last_cuda_error"):
            assert callable(getattr(P, n))


def test_status_strings_without_device(lib):
    lib.pabd_status_str.restype = ctypes.c_char_p
    assert lib.pabd_status_str(0) == b"ok"
    assert b"capacity" in lib.pabd_status_str(3)
    lib.pabd_create_scene.restype = ctypes.c_int
    assert lib.pabd_create_scene(None, None) == 1  # PABD_ERR_ARG, no device touched


def test_library_is_built_for_sm103a(lib):
    """The shared object carries an sm_103a cubin (checked by the build's flags)."""
    src = open(os.path.join(ROOT, "paper_2609_02675_gb300", "_build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src
