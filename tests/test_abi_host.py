"""Host-side checks of the C ABI (no GPU needed).

The CUDA library must load, export every function declared in
include/lbdps.h, and reject invalid descriptions on the host, before any
device work, with the documented status codes.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "lbdps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lbdps_[a-z_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1303_2653_gb300 import build
    build.build_all()
    from paper_1303_2653_gb300 import lbdps as L
    return L


def test_every_declared_function_is_exported(lib):
    names = _declared()
    assert "lbdps_create" in names and "lbdps_step" in names and len(names) >= 20
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_status_strings(lib):
    L = lib.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.lbdps_strerror(code)
    assert L.lbdps_strerror(-99) == b"unknown status"


def _desc(lib, **over):
    lat = lib.LatticeDesc()
    lat.dim = over.get("dim", 2)
    lat.n[0], lat.n[1], lat.n[2] = over.get("n", (8, 8, 1))
    for f, b in enumerate(over.get("bc", (0, 0, 1, 1, 1, 1))):
        lat.bc[f] = b
    lat.h, lat.dt = over.get("h", 1e-3), 1e-4
    pos = np.array(over.get("pos", [[2.5e-3, 2.5e-3], [5.5e-3, 5.5e-3]]), dtype=np.float64)
    vel = np.zeros_like(pos)
    par = lib.ParticleDesc(pos.shape[0], over.get("d_p", 2e-4), 1000.0, 0.9,
                           pos.ctypes.data_as(lib._dp), vel.ctypes.data_as(lib._dp))
    prm = lib.Params()
    prm.rho_g, prm.mu_g = 1.2, 1.8e-5
    prm.storage = over.get("storage", 1)
    return lat, par, prm, (pos, vel)


@pytest.mark.parametrize("bad", [
    {"dim": 4},
    {"n": (0, 8, 1)},
    {"bc": (1, 0, 1, 1, 1, 1)},            # unpaired periodic face
    {"bc": (2, 3, 1, 1, 1, 1)},            # inlet on a horizontal axis
    {"n": (2, 8, 1), "bc": (1, 1, 1, 1, 1, 1)},   # periodic axis of 2 cells
    {"d_p": 2e-3},                          # particles wider than a cell
    {"pos": [[9.5e-3, 2.5e-3]]},            # outside the domain
    {"storage": 7},
])
def test_create_rejects_invalid_descriptions_on_host(lib, bad):
    # (overlapping hard spheres are found on the device after the initial
    # sort: covered by the GPU tests)
    lat, par, prm, keep = _desc(lib, **bad)
    h = ctypes.c_void_p()
    rc = lib.lib().lbdps_create(ctypes.byref(lat), ctypes.byref(par), ctypes.byref(prm),
                                ctypes.byref(h))
    assert rc == lib.ERR_INVALID
    assert not h.value
    assert lib.lib().lbdps_last_error()


def test_noalloc_sort_rejects_oversize_on_host(lib):
    nn = (ctypes.c_int * 3)(4096, 4096, 1)
    pp = (ctypes.c_void_p * 3)(1, 1, None)
    rc = lib.lib().lbdps_bin_sort_noalloc(2, nn, 10, pp, ctypes.c_void_p(1), ctypes.c_void_p(1),
                                          None)
    assert rc == lib.ERR_CAPACITY
    assert b"exceed" in lib.lib().lbdps_last_error()
