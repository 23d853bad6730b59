"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function include/mrf.h declares (no compute calls without a GPU)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1611_06684_gb300 import build
    path = build.build()
    return ct.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared("mrf.h")
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in mrf.h but not exported"


def test_binding_covers_every_symbol():
    from paper_1611_06684_gb300 import mrf as M
    assert set(_declared("mrf.h")) <= set(M.exported_symbols())


def test_host_only_entry_points(lib):
    from paper_1611_06684_gb300 import mrf as M
    M.load()
    opt = M.mrf_options()
    M._lib.mrf_default_options(ct.byref(opt))
    assert opt.use_graphs == 1 and opt.grid_nx == 0
    assert M._lib.mrf_status_string(M.MRF_ENONFINITE) == b"non-finite log-potential"
    # argument validation happens before any device work
    h = ct.c_void_p()
    assert M._lib.mrf_create(ct.byref(h), 10, 17, 1, 0, None, None) == M.MRF_ERANGE
    assert M._lib.mrf_create(ct.byref(h), 0, 4, 1, 0, None, None) == M.MRF_EINVAL
    assert M._lib.mrf_create(None, 10, 4, 1, 0, None, None) == M.MRF_EINVAL
    assert M._lib.mrf_sweep(None, 1, 0) == M.MRF_EINVAL
