"""C-ABI checks that need no GPU: the library loads, exports every declared entry
point, and rejects invalid arguments before touching the device."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(yf_[a-z0-9_]+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def yf():
    from paper_2208_04371_b300 import build
    build.build()
    from paper_2208_04371_b300 import yf as mod
    return mod


def test_library_exports_every_declared_symbol(yf):
    import ctypes
    lib = ctypes.CDLL(yf.library_path())
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared entry point with its own signature
    assert declared <= set(yf.DECLARED)


def test_courant_dt_host_only(yf):
    dt = yf.courant_dt(1e-4, 1e-4, 1e-4, 0.9)
    assert abs(dt - 0.173e-12) < 0.0005e-12


def test_invalid_arguments_are_rejected_without_a_device(yf):
    with pytest.raises(yf.YFError) as e:
        yf.grid_create(2, 10, 10, 1e-6, 1e-6, 1e-6)
    assert e.value.code == yf.E_INVALID
    with pytest.raises(yf.YFError) as e:
        yf.courant_dt(1e-6, 1e-6, 1e-6, 1.2)
    assert e.value.code == yf.E_INVALID


def test_courant_violation_is_unstable(yf):
    lim = yf.courant_dt(1e-6, 1e-6, 1e-6, 1.0)
    with pytest.raises(yf.YFError) as e:
        yf.grid_create(8, 8, 8, 1e-6, 1e-6, 1e-6, dt=1.01 * lim)
    assert e.value.code == yf.E_UNSTABLE
