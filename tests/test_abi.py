"""The C-ABI library loads and exports every entry point include/vls.h declares (no GPU
calls); host-side constants agree bit for bit with the oracle's."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_13168_gb300 import build as libbuild
    from paper_2105_13168_gb300 import vls

    libbuild.build()
    return vls.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "vls.h")).read()
    return sorted(set(re.findall(r"^VLS_API[^(]*?\b(vls_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_api():
    names = declared_symbols()
    assert "vls_detect" in names and "vls_detect_batch" in names and "vls_result_reeb" in names
    assert len(names) >= 19


def test_library_exports_every_declared_symbol(lib):
    import ctypes

    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_exports():
    from paper_2105_13168_gb300 import vls

    assert sorted(vls.EXPORTS) == declared_symbols()


def test_constants_bitwise_equal_oracle(lib):
    import oracle
    from paper_2105_13168_gb300 import vls

    a = vls.vls_constants()
    b = oracle.constants()
    for k in ("eta", "lbar", "dt", "s"):
        assert a[k] == b[k], k
    o = vls.vls_default_options()
    oo = oracle.default_options()
    for k in ("mu", "e", "a", "w", "dt_factor", "eps0", "theta_iso"):
        assert getattr(o, k) == getattr(oo, k), k


def test_status_strings(lib):
    for s in range(13):
        assert lib.vls_status_string(s)
