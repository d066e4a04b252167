"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/dw.h declares (no compute call: runs without a GPU)."""

import ctypes
import os
import re

from paper_2112_01852_gb300 import build, dw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(dw_[a-z_A-Z0-9]+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dw_create_lattice", "dw_load_gauge", "dw_apply_Dhop", "dw_apply_D",
                     "dw_apply_Ddag", "dw_apply_DdagD", "dw_cg_solve"):
        assert required in names
    assert names == set(dw.SYMBOLS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    # the Python binding resolves every symbol with its signature
    dw.load_library()


def test_create_lattice_checks_its_arguments_before_any_device_call():
    # argument errors come back as DW_ERR_ARG with a message, before the call
    # touches a device (so this runs without a GPU): zero extents, an unknown
    # kind, and a Moebius b of zero (the D kernels divide c by b)
    import pytest
    build.build()
    cases = [((4, 0, 4, 4), 4, dw.DW_MOBIUS, 1.5, 0.5),
             ((4, 4, 4, 4), 0, dw.DW_MOBIUS, 1.5, 0.5),
             ((4, 4, 4, 4), 4, 7, 1.5, 0.5),
             ((4, 4, 4, 4), 4, dw.DW_MOBIUS, 0.0, 0.5),
             ((4, 4, 4, 4), 4, dw.DW_MOBIUS, float("nan"), 0.5)]
    for dims, Ls, kind, b, c in cases:
        with pytest.raises(dw.DWError) as e:
            dw.dw_create_lattice(dims, Ls, kind, 1.8, b, c, dw.DW_F32)
        assert e.value.code == dw.DW_ERR_ARG, (dims, Ls, kind, b)
        assert dw.dw_last_error()
