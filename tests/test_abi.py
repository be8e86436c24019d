"""The C-ABI library builds, loads and exports every symbol its headers
declare (no compute calls: this runs without a GPU)."""
import ctypes
import subprocess

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
