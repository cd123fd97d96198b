"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/apo.h declares (no GPU needed: no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(apo4?_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    import paper_2401_04576_gb300.build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    names = _declared("apo.h") + _declared("apo_diag.h") + _declared("apo4.h")
    assert len(names) >= 13 and "apo4_solve_batch" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_opts_default_and_errors_without_gpu():
    from paper_2401_04576_gb300 import apo
    o = apo.solve_opts()
    assert o.max_tracks == 1 and o.min_votes == 0 and abs(o.mask_sigma - 150e-6) < 1e-18
    assert all(o.precision[i] == apo.F64 for i in range(apo.MAX_LEVELS + 1))
    L = apo.lib()
    assert L.apo_geometry_create(None, None, None) == apo.APO_EINVAL
    assert b"NULL" in L.apo_last_error()


def test_four_d_defaults_and_errors_without_gpu():
    from paper_2401_04576_gb300 import apo
    o = apo.four_opts()
    assert o.n_iter == 3 and o.precision == apo.F64 and abs(o.p_gev - 0.105) < 1e-15
    assert [o.n[1][a] for a in range(4)] == [90, 90, 40, 20]
    L = apo.lib()
    assert L.apo4_chamber_create(None, None) == apo.APO_EINVAL
