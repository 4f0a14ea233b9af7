"""CPU checks of the C ABI library: it builds for sm_103a, loads, and exports
every function declared in include/*.h (no compute calls: there is no GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mfc_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mfc_init", "mfc_set_state", "mfc_rhs", "mfc_step", "mfc_cfl_dt",
                     "mfc_get_state", "mfc_finalize", "mfc_last_error"):
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    import paper_2305_09163_gb300 as m
    path = m.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_c_abi():
    import paper_2305_09163_gb300 as m
    for n in _declared():
        assert hasattr(m, n), n


def test_invalid_init_arguments_are_rejected_without_a_gpu():
    """Argument validation happens before any CUDA call."""
    import paper_2305_09163_gb300 as m
    bad = [
        dict(n=(2, 1, 1)),                      # fewer than 3 cells on an active axis
        dict(n=(8, 1, 4)),                      # inactive middle axis
        dict(bc=(0, 1, 1, 1, 1, 1)),            # periodic on one side only
        dict(gamma=(1.0,), pi_inf=(0.0,)),      # gamma must exceed 1
        dict(gamma=(1.4, 1.4, 1.4, 1.4), pi_inf=(0,) * 4),  # at most 3 fluids
        dict(precision=7),
    ]
    for over in bad:
        kw = dict(n=(8, 1, 1), lo=(0, 0, 0), hi=(1, 1, 1), bc=(1,) * 6, gamma=(1.4,), pi_inf=(0.0,),
                  precision=0)
        kw.update(over)
        with pytest.raises(m.MFCError) as ei:
            m.mfc_init(kw["n"], kw["lo"], kw["hi"], kw["bc"], kw["gamma"], kw["pi_inf"], kw["precision"], None)
        assert ei.value.status == m.MFC_ERR_ARG
