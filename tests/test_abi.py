"""The C ABI library builds, loads without a GPU and exports every entry point
that include/acat.h declares; argument checks that need no device work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_01416_gb300 import build as B
    B.build()
    from paper_2007_01416_gb300 import acat
    return acat.lib()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(acat_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("acat_create", "acat_step", "acat_run", "acat_destroy", "acat_status"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\sT\s(\w+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)  # resolvable through dlsym


def test_params_struct_matches_header(lib):
    from paper_2007_01416_gb300 import acat
    p = acat.default_params()
    assert p.P == 2 and p.ny == 1 and p.tau_factorial == 1
    assert abs(p.gamma - 1.4) < 1e-15 and p.eps == 1e-12 and p.psi_tol == 0.1
    # 11 ints, 4 bytes of padding to the 8-byte alignment of the doubles, 10 doubles
    assert ctypes.sizeof(acat.acat_params) == 11 * 4 + 4 + 10 * 8
    assert acat.acat_params.gamma.offset == 48 and p.rect_2d == 0


@pytest.mark.parametrize("bad", [dict(P=0), dict(P=5), dict(nx=3, P=2), dict(flux=9), dict(cfl=0.0),
                                 dict(bc=7), dict(psi_tol=1.0), dict(eps=-1.0),
                                 dict(flux=2, gamma=1.0), dict(x1=-1.0), dict(psi2_mod=2), dict(lo_flux=3),
                                 dict(rect_2d=2)])
def test_create_rejects_bad_params_without_device(lib, bad):
    # validation runs before any CUDA call
    from paper_2007_01416_gb300 import acat
    p = acat.make_params(**bad)
    h = ctypes.c_void_p()
    rc = lib.acat_create(ctypes.byref(p), ctypes.byref(h))
    assert rc == -1 and not h.value


def test_strerror(lib):
    from paper_2007_01416_gb300 import acat
    assert acat.strerror(0) == "ok"
    assert "invalid" in acat.strerror(-1)
    assert acat.strerror(-999) == "unknown error"


@pytest.mark.parametrize("kw", [dict(nx=(1 << 30) + 1), dict(flux=3, P=2, nx=1 << 16, ny=(1 << 15) + 1)])
def test_create_rejects_too_large_without_device(lib, kw):
    from paper_2007_01416_gb300 import acat
    p = acat.make_params(**kw)
    h = ctypes.c_void_p()
    assert lib.acat_create(ctypes.byref(p), ctypes.byref(h)) == -6 and not h.value
