"""Host-side checks of the C ABI: the library loads, exports every entry point include/qmmm.h
declares, and rejects invalid input before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2408_03273_gb300 as q
from paper_2408_03273_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "qmmm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qmmm_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = q.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    # and the binding marshals every one of them under the same name
    assert sorted(q.EXPORTS) == names
    for n in names:
        assert callable(getattr(q, n)), n


def test_error_strings():
    assert q.qmmm_strerror(0) == "ok"
    for code in (-1, -2, -3, -4, -5, -6):
        assert q.qmmm_strerror(code) != "unknown error"


def _tiny_args():
    return dict(atom_xyz=np.zeros((1, 3)), atom_Z=[1.0], shell_atom=[0], shell_l=[0], shell_nprim=[1],
                shell_prim_offset=[0], prim_exp=[1.0], prim_coeff=[1.0], mm_xyz=np.array([[3.0, 0, 0]]),
                mm_q=[0.5], mm_sigma=[0.3], box=[20.0, 20.0, 20.0], cutoff=8.0, ewald_alpha=0.3)


@pytest.mark.parametrize("field,value,code", [
    ("shell_l", [4], -5),            # g shells are not supported
    ("shell_nprim", [17], -5),       # more than 16 primitives
    ("prim_exp", [-1.0], -1),        # non-positive exponent
    ("shell_atom", [3], -1),         # shell on a missing atom
    ("box", [0.0, 20.0, 20.0], -1),  # degenerate box
    ("cutoff", -1.0, -1),
    ("ewald_alpha", 0.0, -1),
    ("mm_q", [float("nan")], -1),
])
def test_create_rejects_invalid_input_on_host(field, value, code):
    # all of these are caught before any CUDA call, so they run on a machine without a GPU
    args = _tiny_args()
    args[field] = value
    if field == "shell_nprim":
        args["prim_exp"] = [1.0] * 17
        args["prim_coeff"] = [1.0] * 17
    with pytest.raises(q.QMMMError) as ei:
        q.qmmm_create(**args)
    assert ei.value.code == code


def test_null_handle_is_an_argument_error():
    L = q.load()
    assert L.qmmm_vpot(None, None, None) == -1
    assert L.qmmm_forces(None, None, None, None, None) == -1
    assert L.qmmm_nao(None) == -1
    out = (ctypes.c_double * 2)()
    assert L.qmmm_last_timing(None, out) == -1


def test_binding_rejects_wrong_dtype():
    with pytest.raises(TypeError):
        _lib._ptr(np.zeros(3, dtype=np.float32))
    with pytest.raises(TypeError):
        _lib._ptr(np.zeros((3, 3))[:, 0])
