"""The C-ABI library builds, loads and exports every symbol its headers
declare, and its host-side argument checks answer before any CUDA call (no
compute calls: this runs without a GPU)."""
import ctypes
import subprocess

import pytest

from paper_2310_03921_gb300 import build as B
from paper_2310_03921_gb300 import gap


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    L = ctypes.CDLL(path)
    names = gap.exported_symbols()
    assert "gap_predict" in names and "gap_descriptor" in names and "gap_assemble_knm" in names
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T gap_" in line}
    assert exported == set(names)


def test_binding_loads_and_reports_errors_without_a_gpu():
    L = gap.lib()
    p = gap.SoapParams(0, 4, 5.0, 1.0, 0.5, 1.0, 1, 0, None)   # n_max = 0 is invalid
    h = ctypes.c_void_p()
    st = L.gap_soap_create(ctypes.byref(p), ctypes.byref(h))
    assert st == -1 and b"n_max" in L.gap_last_error()
    assert L.gap_soap_destroy(None) == 0


@pytest.mark.parametrize("args,status,msg", [
    ((5, 5, 5.0, 1.0, 0.5, 1.0, 1, 0, None), -6, b"no compiled kernel"),
    ((6, 11, 5.0, 1.0, 0.5, 1.0, 1, 0, None), -1, b"l_max"),
    ((13, 4, 5.0, 1.0, 0.5, 1.0, 1, 0, None), -1, b"n_max"),
    ((6, 4, 5.0, 6.0, 0.5, 1.0, 1, 0, None), -1, b"cutoff_transition_width"),
    ((6, 4, 5.0, 1.0, 0.0, 1.0, 1, 0, None), -1, b"atom_sigma"),
    ((6, 4, 5.0, 1.0, 0.5, 1.0, 0, 0, None), -1, b"n_species"),
    ((6, 4, 5.0, 1.0, 0.5, 1.0, 2, 1, None), -1, b"mix_w"),
])
def test_descriptor_parameters_are_checked_on_the_host(args, status, msg):
    """gap_soap_create rejects bad parameters and shapes without a compiled
    kernel before it touches the GPU (GAP_EINVAL, GAP_EUNSUPPORTED)."""
    L = gap.lib()
    h = ctypes.c_void_p()
    assert L.gap_soap_create(ctypes.byref(gap.SoapParams(*args)), ctypes.byref(h)) == status
    assert msg in L.gap_last_error() and not h.value


def test_null_handles_are_rejected():
    L = gap.lib()
    d = ctypes.c_double(1.0)
    assert L.gap_model_create(None, 1, None, None, None, d, ctypes.c_double(4.0), None, None) == -1
    assert L.gap_predict(None, None, 1, None, None, None, None, None) == -1
    assert L.gap_assemble_knm(None, None, 1, None, None) == -1
    assert L.gap_model_destroy(None) == 0 and L.gap_step_graph_destroy(None) == 0


def test_profile_stage_names():
    L = gap.lib()
    L.gap_profile_stage_name.restype = ctypes.c_char_p
    names = [L.gap_profile_stage_name(k) for k in range(L.gap_profile_stages())]
    assert all(names) and len(set(names)) == len(names)
    for s in (b"neighbours", b"knm_gemm", b"knm_jacobian", b"solve_block"):
        assert s in names
