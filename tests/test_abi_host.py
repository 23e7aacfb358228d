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
    lat.h, lat.dt = over.get("h", 1e-3), over.get("dt", 1e-4)
    inlet = None
    if "inlet_u" in over:
        inlet = np.ascontiguousarray(over["inlet_u"], dtype=np.float64)
        lat.inlet_u = inlet.ctypes.data_as(lib._dp)
    pos = np.array(over.get("pos", [[2.5e-3, 2.5e-3], [5.5e-3, 5.5e-3]]), dtype=np.float64)
    vel = np.zeros_like(pos)
    par = lib.ParticleDesc(over.get("np", pos.shape[0]), over.get("d_p", 2e-4),
                           over.get("rho_s", 1000.0), over.get("e", 0.9),
                           None if over.get("null_arrays") else pos.ctypes.data_as(lib._dp),
                           None if over.get("null_arrays") else vel.ctypes.data_as(lib._dp))
    par.recirculate = over.get("recirculate", 0)
    par.collision_model = over.get("collision_model", 0)
    par.dem_kn = over.get("dem_kn", 0.0)
    par.dem_mu = over.get("dem_mu", 0.0)
    par.dem_gamma_t = over.get("dem_gamma_t", 0.0)
    prm = lib.Params()
    prm.rho_g, prm.mu_g = over.get("rho_g", 1.2), over.get("mu_g", 1.8e-5)
    for a, u in enumerate(over.get("u0", (0.0, 0.0, 0.0))):
        prm.u0[a] = u
    prm.cs_smag = over.get("cs_smag", 0.0)
    prm.superficial_mode = over.get("superficial_mode", 0)
    prm.storage = over.get("storage", 1)
    return lat, par, prm, (pos, vel, inlet)


# Units of the base description: h = 1 mm, dt = 0.1 ms, particles of 0.2 mm
# and 1000 kg/m^3 (m_p = 4.19e-9 kg), air: tau = 0.5045, d/h = 0.2.
_SOFT = {"collision_model": 1, "dem_kn": 0.01}   # a pair contact lasts 14 steps


@pytest.mark.parametrize("bad,msg", [
    ({"dim": 4}, "dim must be 2 or 3"),
    ({"n": (0, 8, 1)}, "must be positive"),
    ({"n": (50000, 50000, 1)}, "lattice too large"),
    ({"bc": (0, 0, 7, 3, 1, 1)}, "unknown face type"),
    ({"bc": (1, 0, 1, 1, 1, 1)}, "must come in pairs"),
    ({"bc": (2, 3, 1, 1, 1, 1)}, "only on the vertical axis"),
    ({"bc": (0, 0, 2, 2, 1, 1)}, "at most one inlet"),
    ({"n": (2, 8, 1), "bc": (1, 1, 1, 1, 1, 1)}, "at least 3 cells"),
    ({"dt": -1e-4}, "h and dt must be positive"),
    ({"np": -1}, "bad particle count"),
    ({"null_arrays": True}, "NULL particle arrays"),
    ({"e": 1.5}, "bad particle properties"),
    ({"rho_s": 0.0}, "bad particle properties"),
    ({"d_p": 2e-3}, "must not exceed h"),
    ({"recirculate": 2}, "bad recirculate"),
    ({"recirculate": 1}, "inlet below and the outlet above"),
    ({"collision_model": 5}, "bad collision_model"),
    ({"collision_model": 1}, "need dem_kn > 0"),
    ({**_SOFT, "e": 0.0}, "need e > 0"),
    ({**_SOFT, "dem_mu": -0.5}, "finite and >= 0"),
    ({"dem_mu": 0.5, "dem_gamma_t": 1e-7}, "friction needs soft spheres"),
    ({"mu_g": 0.0}, "bad gas properties"),
    ({"storage": 7}, "bad storage"),
    ({"cs_smag": -0.1}, "bad Smagorinsky"),
    ({"superficial_mode": 3}, "bad superficial_mode"),
    ({"mu_g": 1e-30}, "tau must exceed 1/2"),
    ({**_SOFT, "dem_kn": 1e3}, "too stiff"),
    ({**_SOFT, "dem_mu": 0.5, "dem_gamma_t": 1.0}, "dem_gamma_t too large"),
    ({"u0": (0.0, 5.0, 0.0)}, "|u0| must be below 0.3"),
    ({"bc": (0, 0, 2, 3, 1, 1), "inlet_u": np.tile([0.0, 5.0], (8, 1))}, "inlet |u| must be"),
    ({"d_p": 1e-5}, "too small for the cell"),
    ({"pos": [[9.5e-3, 2.5e-3]]}, "outside the domain"),
])
def test_create_rejects_invalid_descriptions_on_host(lib, bad, msg):
    # every check of lbdps_create runs on the host before the first CUDA call
    # (overlapping hard spheres are found on the device after the initial
    # sort: covered by the GPU tests)
    lat, par, prm, keep = _desc(lib, **bad)
    h = ctypes.c_void_p()
    rc = lib.lib().lbdps_create(ctypes.byref(lat), ctypes.byref(par), ctypes.byref(prm),
                                ctypes.byref(h))
    assert rc == lib.ERR_INVALID
    assert not h.value
    assert msg.encode() in lib.lib().lbdps_last_error()


def test_noalloc_sort_rejects_oversize_on_host(lib):
    nn = (ctypes.c_int * 3)(4096, 4096, 1)
    pp = (ctypes.c_void_p * 3)(1, 1, None)
    rc = lib.lib().lbdps_bin_sort_noalloc(2, nn, 10, pp, ctypes.c_void_p(1), ctypes.c_void_p(1),
                                          None)
    assert rc == lib.ERR_CAPACITY
    assert b"exceed" in lib.lib().lbdps_last_error()
