"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/lu.h, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import pytest

import paper_1611_06365_gb300 as lu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    lu.build()
    return lu.lib()


def declared_functions():
    with open(os.path.join(ROOT, "include", "lu.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lu_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "lu_factor" in names and "lu_solve_mixed" in names
    for name in names:
        assert hasattr(L, name), name
        assert isinstance(getattr(L, name), ctypes._CFuncPtr)


def test_status_strings(L):
    assert lu.lu_status_string(0) == "success"
    assert "timeout" in lu.lu_status_string(lu.LU_ERR_TIMEOUT) or "wait" in lu.lu_status_string(lu.LU_ERR_TIMEOUT)
    assert "argument" in lu.lu_status_string(-3)
    assert "sm_103a" in lu.lu_version()


def test_argument_errors_return_minus_i(L):
    f = L.lu_factor
    dummy = ctypes.c_void_p(16)
    assert f(7, 4, dummy, 4, dummy, dummy, None, None) == -1        # bad dtype
    assert f(0, -1, dummy, 4, dummy, dummy, None, None) == -2       # n < 0
    assert f(0, 4, None, 4, dummy, dummy, None, None) == -3         # A null
    assert f(0, 4, dummy, 3, dummy, dummy, None, None) == -4        # lda < n
    assert f(0, 4, dummy, 4, None, dummy, None, None) == -5         # ipiv null
    assert f(0, 4, dummy, 4, dummy, None, None, None) == -6         # info null
    o = lu.LuOpts(0, 0, 17, 0, 0, 0)                                # panel_ctas > 16
    assert f(0, 4, dummy, 4, dummy, dummy, ctypes.byref(o), None) == -7
    o = lu.LuOpts(0, 0, 0, 0, lu.LU_UPDATE_BF16, 0)                 # BF16 update needs FP32
    assert f(0, 4, dummy, 4, dummy, dummy, ctypes.byref(o), None) == -7
    o = lu.LuOpts(0, 0, 0, 2, 0, 0, 0, 0, 0, 1)                     # early termination needs depth 1
    assert f(0, 4, dummy, 4, dummy, dummy, ctypes.byref(o), None) == -7
    assert L.lu_last_panel_widths(None, 0) >= -1                    # -1 until a factorization ran
    s = L.lu_solve
    assert s(0, 4, -1, dummy, 4, dummy, dummy, 4, None) == -3
    assert s(0, 4, 1, dummy, 4, dummy, dummy, 2, None) == -8
    assert L.lu_solve_mixed(-1, 1, dummy, 1, dummy, 1, dummy, 1, None, None, None) == -1
    assert L.lu_solve_mixed(4, 1, dummy, 4, dummy, 4, dummy, 3, None, None, None) == -8
    assert L.lu_factor_batched(0, 3, dummy, dummy, dummy, dummy, dummy, 2000, None, None) == -8
    assert L.lu_trailing_update(1, 4, 4, 300, dummy, 4, dummy, 300, dummy, 4, None) == -4


def test_workspace_sizes(L):
    assert lu.lu_workspace_size("solve", 1000, 1, lu.LU_F64) > 1000 * 8
    assert lu.lu_workspace_size("mixed", 1000, 1, lu.LU_F64) > 1000 * 1000 * 4
    assert lu.lu_workspace_size("nothing", 10, 1, lu.LU_F64) == 0


def test_colmajor_helpers():
    torch = pytest.importorskip("torch")
    M = torch.arange(12, dtype=torch.float64).view(3, 4)
    T = lu.to_colmajor(M, ld=5)
    assert T.shape == (4, 5) and float(T[1, 2]) == float(M[2, 1])
    assert torch.equal(lu.from_colmajor(T, 3), M)


def test_binding_struct_layouts_match_the_library(L):
    """Every public struct the binding mirrors has the size the library was built with
    (a field added on one side only would shift the fields after it)."""
    for name, cls in (("lu_opts", lu.LuOpts), ("lu_mixed_opts", lu.MixedOpts), ("lu_mixed_report", lu.MixedReport),
                      ("lu_tune_result", lu.TuneResult), ("lu_trace_event", lu.TraceEvent),
                      ("lu_cta_event", lu.CtaEvent)):
        assert L.lu_abi_size(name.encode()) == ctypes.sizeof(cls), name
    assert L.lu_abi_size(b"no_such_struct") == 0
