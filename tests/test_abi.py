"""The C ABI library builds, loads and exports every entry point of include/dbfft.h (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "dbfft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dbfft_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ["dbfft_create", "dbfft_apply", "dbfft_solve_increment", "dbfft_homogenized_stress",
              "dbfft_homogenized_tangent", "dbfft_adjoint", "dbfft_destroy", "dbfft_last_error"]:
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_1905_12725_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    from paper_1905_12725_gb300 import dbfft
    assert sorted(dbfft.EXPORTS) == sorted(n for n in _declared()), "binding and header disagree"
    lib.dbfft_status_string.restype = ctypes.c_char_p
    assert lib.dbfft_status_string(5) == b"DBFFT_E_NOT_CONVERGED"


def test_binding_constants_match_the_header_enums():
    """Every `DBFFT_NAME = value` of the header's enums that the binding defines has the same value."""
    txt = open(os.path.join(ROOT, "include", "dbfft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    pairs = dict((n, int(v)) for n, v in re.findall(r"\b(DBFFT_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt))
    from paper_1905_12725_gb300 import dbfft
    shared = [n for n in pairs if hasattr(dbfft, n)]
    for n in ["DBFFT_SMALL", "DBFFT_FINITE", "DBFFT_FP64", "DBFFT_MIXED", "DBFFT_ISO_ELASTIC", "DBFFT_NEO_HOOKE",
              "DBFFT_CP_FCC_POWERLAW", "DBFFT_SVK", "DBFFT_CP_FCC_FINITE"]:
        assert n in shared, n
    for n in shared:
        assert getattr(dbfft, n) == pairs[n], n
    assert dbfft.cp_phases([[1.0, 0, 0, 0]], finite=True)[0].model == pairs["DBFFT_CP_FCC_FINITE"]
