"""C-ABI checks that need no GPU: the library loads, exports every entry point
the header declares, and rejects invalid arguments before touching the device."""

import ctypes
import os
import re

import pytest

from paper_2609_18026_b300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_names():
    txt = open(os.path.join(ROOT, "include", "mlx.h")).read()
    return sorted(set(re.findall(r"\b(mlx_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_18026_b300 import build
    build.build()
    return B.load()


def test_exports_every_declared_symbol(lib):
    names = _header_names()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.EXPORTS)


def test_strerror(lib):
    assert lib.mlx_strerror(0) == b"ok"
    assert lib.mlx_strerror(-1) == b"invalid argument"
    assert lib.mlx_strerror(-5) == b"call out of order"


@pytest.mark.parametrize("kw", [
    dict(nr=1, nphi=8, nz=1, ell=1.0), dict(nr=8, nphi=12, nz=1, ell=1.0),
    dict(nr=8, nphi=8, nz=3, ell=1.0), dict(nr=8, nphi=8, nz=1, ell=0.0), dict(nr=8, nphi=1024, nz=1, ell=1.0),
    dict(nr=8, nphi=8, nz=1, ell=1.0, lz=-1.0), dict(nr=8, nphi=8, nz=1, ell=1.0, precision=7),
    dict(nr=8, nphi=8, nz=1, ell=1.0, nphi_c=6), dict(nr=8, nphi=8, nz=4, ell=1.0, nz_c=4),
    dict(nr=8, nphi=8, nz=1, ell=1.0, nr_c=9), dict(nr=4, nphi=16, nz=1, ell=1.0, nphi_c=8),
    dict(nr=8, nphi=8, nz=1, ell=1.0, chop_policy=3), dict(nr=4, nphi=8, nz=1, ell=1.0, chop_policy=2)])
def test_create_rejects_invalid(lib, kw):
    # chops one past the Nyquist-keeping bounds (M = Nphi/2 + 1, Kz = Nz/2 + 1), an
    # unknown policy, and a Nyquist chop whose M = 5 exceeds Nc = 4
    p = B.Params(kw["nr"], kw["nphi"], kw["nz"], kw.get("nr_c", 0), kw.get("nphi_c", 0),
                 kw.get("nz_c", 0), kw["ell"], kw.get("lz", 1.0), kw.get("precision", 0),
                 kw.get("chop_policy", 0))
    h = ctypes.c_void_p(123)
    assert lib.mlx_create(ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert not h.value


def test_null_arguments(lib):
    assert lib.mlx_create(None, None, None) == -1
    assert lib.mlx_query(None, None) == -1
    assert lib.mlx_destroy(None) == -1
    assert lib.mlx_forward(None, None, None, None) == -1
    assert lib.mlx_advance(None, 0, None, 0, None, None, 1, 1, None) == -1
