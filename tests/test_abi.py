"""The C ABI library loads, exports every symbol include/tileqr.h declares,
and its host-only entry points (sizes, argument checks, error text) behave;
no GPU is needed for any of this."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    return tileqr.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "tileqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tileqr_[A-Za-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_0709_1272_gb300 import tileqr
    assert sorted(tileqr.EXPORTED) == names


def test_workspace_size_layout(lib):
    from paper_0709_1272_gb300 import tileqr
    for (m, n, nb, ib) in [(512, 512, 64, 16), (16384, 16384, 128, 32), (262144, 512, 128, 32),
                           (1000, 700, 128, 16), (1, 1, 64, 16)]:
        b = tileqr.tileqr_workspace_size(m, n, nb, ib)
        p, q = -(-m // nb), -(-n // nb)
        tiles = p * q * nb * nb * 8
        assert b >= tiles + p * q * ib * nb * 8
        assert b % 256 == 0
        # scheduler state stays small next to the tiles
        assert b - tiles - p * q * ib * nb * 8 <= 0.01 * tiles + 4 * 2**20


def test_argument_errors(lib):
    sz = ctypes.c_size_t(0)
    assert lib.tileqr_workspace_size(-1, 4, 64, 16, 0, ctypes.byref(sz)) == -1
    assert lib.tileqr_workspace_size(4, -1, 64, 16, 0, ctypes.byref(sz)) == -2
    assert lib.tileqr_workspace_size(4, 4, 0, 16, 0, ctypes.byref(sz)) == -5
    assert lib.tileqr_workspace_size(4, 4, 64, 24, 0, ctypes.byref(sz)) == -6
    assert lib.tileqr_workspace_size(4, 4, 64, 128, 0, ctypes.byref(sz)) == -6
    from paper_0709_1272_gb300 import tileqr
    d = tileqr.tileqr_desc()
    # illegal lda is reported before any device work
    rc = lib.tileqr_factor(10, 10, ctypes.c_void_p(1), 5, 64, 16, 0, 0, 0, None, 0, None, ctypes.byref(d))
    assert rc == -4
    rc = lib.tileqr_factor(10, 10, ctypes.c_void_p(1), 10, 64, 16, 0, 7, 0, None, 0, None, ctypes.byref(d))
    assert rc == -8
    # unbuilt (nb, ib): explicit error, never a fallback
    rc = lib.tileqr_factor(10, 10, ctypes.c_void_p(1), 10, 48, 16, 0, 0, 0, None, 0, None, ctypes.byref(d))
    assert rc == tileqr.TILEQR_ERR_UNSUPPORTED
    rc = lib.tileqr_factor(10, 10, ctypes.c_void_p(1), 10, 64, 16, 0, 0, 0, None, 0, None, ctypes.byref(d))
    assert rc == tileqr.TILEQR_ERR_WORKSPACE


def test_strerror(lib):
    from paper_0709_1272_gb300 import tileqr
    assert "watchdog" in tileqr.strerror(tileqr.TILEQR_ERR_TIMEOUT)
    assert tileqr.strerror(0) == "success"
    assert tileqr.strerror(-3) == "illegal argument"
