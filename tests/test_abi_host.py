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


def _create(lib, **over):
    lat, par, prm, keep = _desc(lib, **over)
    h = ctypes.c_void_p()
    rc = lib.lib().lbdps_create(ctypes.byref(lat), ctypes.byref(par), ctypes.byref(prm),
                                ctypes.byref(h))
    if h.value:
        lib.lib().lbdps_destroy(h)
    return rc, lib.lib().lbdps_last_error()


def test_domain_check_at_the_fp64_boundary(lib):
    # a particle is inside when its position in lattice units, the correctly
    # rounded FP64 quotient x / h, lies in [0, n); the host check skips the
    # division for coordinates well inside, so probe the exact edge: the
    # smallest x whose quotient reaches n is rejected, the next double below
    # passes the host check (what follows needs a device)
    h, n = 1e-3, 8
    x = n * h
    while x / h >= n:
        x = np.nextafter(x, 0.0)
    edge = np.nextafter(x, np.inf)
    assert edge / h >= n and x / h < n
    rc, msg = _create(lib, pos=[[edge, 2.5e-3]])
    assert rc == lib.ERR_INVALID and b"particle 0 lies outside the domain on axis 0" in msg
    rc, msg = _create(lib, pos=[[x, 2.5e-3]])
    assert b"outside the domain" not in msg
    rc, msg = _create(lib, pos=[[2.5e-3, -0.0]])   # -0 / h = -0 >= 0: inside
    assert b"outside the domain" not in msg


def test_domain_check_reports_the_first_particle_outside(lib):
    # the smallest index in (particle, axis) order, as one loop in index
    # order finds it, whichever host thread meets which particle first
    npart = 300000
    pos = np.full((npart, 2), 2.5e-3)
    pos[:, 0] = np.linspace(0.5e-3, 7.5e-3, npart)
    pos[123457, 1] = -1e-300
    pos[200001, 0] = 9e-3
    pos[250000, 1] = 8e-3
    rc, msg = _create(lib, pos=pos)
    assert rc == lib.ERR_INVALID
    assert b"particle 123457 lies outside the domain on axis 1" in msg


def test_noalloc_sort_rejects_oversize_on_host(lib):
    nn = (ctypes.c_int * 3)(4096, 4096, 1)
    pp = (ctypes.c_void_p * 3)(1, 1, None)
    rc = lib.lib().lbdps_bin_sort_noalloc(2, nn, 10, pp, ctypes.c_void_p(1), ctypes.c_void_p(1),
                                          None)
    assert rc == lib.ERR_CAPACITY
    assert b"exceed" in lib.lib().lbdps_last_error()


def test_noalloc_sort_rejects_negative_count_on_host(lib):
    # a negative particle count is an invalid argument, not a capacity error
    nn = (ctypes.c_int * 3)(8, 8, 1)
    pp = (ctypes.c_void_p * 3)(1, 1, None)
    rc = lib.lib().lbdps_bin_sort_noalloc(2, nn, -5, pp, ctypes.c_void_p(1), ctypes.c_void_p(1),
                                          None)
    assert rc == lib.ERR_INVALID
    assert b"bad arguments" in lib.lib().lbdps_last_error()


def test_handle_calls_reject_null_arguments_on_host(lib):
    # every call on a bed or a server answers LBDPS_ERR_INVALID for a NULL
    # handle (or a NULL output) without touching the device
    L = lib.lib()
    calls = {
        "lbdps_step": (None, 1),
        "lbdps_step_monitored": (None, 1, None),
        "lbdps_step_profiled": (None, 1, None, 0, None),
        "lbdps_sync": (None,),
        "lbdps_fields": (None, 1, 0, None, 0),
        "lbdps_particles": (None, 0, None, None, 0),
        "lbdps_set_particles": (None, 0, None, None),
        "lbdps_particle_spin": (None, 0, None, 0),
        "lbdps_set_particle_spin": (None, None, 0),
        "lbdps_populations": (None, None, 0),
        "lbdps_set_populations": (None, None, 0),
        "lbdps_particle_diag": (None, 0, None, 0),
        "lbdps_collide_particles": (None, None, 0, None),
        "lbdps_stats": (None, None),
        "lbdps_health": (None, None),
        "lbdps_constants": (None, None, 0),
        "lbdps_shape": (None, None, None, None, None),
        "lbdps_save": (None, None, 0, None),
        "lbdps_load": (None, None, 0),
        "lbdps_record_event": (None, None),
        "lbdps_bubbles": (None, 0.85, 0, None),
        "lbdps_set_inlet": (None, None),
        "lbdps_check_guards": (None, None),
        "lbdps_server_submit": (None, None, None, None, 1, 0, None),
        "lbdps_server_poll": (None, 0.0, None, 0, None),
        "lbdps_server_load": (None, None, None, None),
        "lbdps_server_take": (None, 1, None),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == lib.ERR_INVALID, name
        assert L.lbdps_last_error(), name
    L.lbdps_destroy(None)
    L.lbdps_server_destroy(None)


def test_empty_server_on_host(lib):
    # creating a server reserves nothing on the device: bad limits are
    # rejected, an empty server reports no load, and taking an unknown
    # request fails cleanly
    L = lib.lib()
    s = ctypes.c_void_p()
    for budget, active, tick in ((0, 4, 8), (1 << 30, 0, 8), (1 << 30, 4, 0)):
        assert L.lbdps_server_create(budget, active, tick, ctypes.byref(s)) == lib.ERR_INVALID
    assert L.lbdps_server_create(1 << 30, 4, 8, ctypes.byref(s)) == lib.OK and s.value
    q, a, used = ctypes.c_int(-1), ctypes.c_int(-1), ctypes.c_size_t(7)
    assert L.lbdps_server_load(s, ctypes.byref(q), ctypes.byref(a), ctypes.byref(used)) == lib.OK
    assert (q.value, a.value, used.value) == (0, 0, 0)
    h = ctypes.c_void_p(1)
    assert L.lbdps_server_take(s, 12345, ctypes.byref(h)) == lib.ERR_INVALID
    assert not h.value
    assert b"no kept result" in L.lbdps_last_error()
    L.lbdps_server_destroy(s)


def test_memory_estimate_on_host(lib):
    # lbdps_memory_estimate does no device work: it validates like
    # lbdps_create and counts the bytes of every buffer of the bed
    L = lib.lib()

    def est(**over):
        lat, par, prm, keep = _desc(lib, **over)
        out = ctypes.c_size_t(0)
        rc = L.lbdps_memory_estimate(ctypes.byref(lat), ctypes.byref(par), ctypes.byref(prm),
                                     ctypes.byref(out))
        return rc, out.value

    ncell, q = 64 * 64, 9
    big = {"n": (64, 64, 1), "h": 1e-3}
    rc64, b64 = est(**big, storage=0)
    rc32, b32 = est(**big, storage=1)
    rc16, b16 = est(**big, storage=2)
    rcbf, bbf = est(**big, storage=3)
    assert (rc64, rc32, rc16, rcbf) == (lib.OK,) * 4
    # two population buffers of q values per cell, and more (ghost layer)
    assert b64 - b32 >= 2 * q * ncell * 4
    assert b32 - b16 >= 2 * q * ncell * 2
    assert b16 == bbf
    # the particle arrays grow with the particle count
    # (each buffer rounded up to 256 B: 2 and 200 particles differ)
    grid = [[(i + 0.5) * 1e-3, (j + 0.5) * 1e-3] for i in range(20) for j in range(10)]
    rc, b32_200 = est(**big, storage=1, pos=grid)
    assert rc == lib.OK and b32_200 > b32
    # the same validation as create
    rc, _ = est(storage=7)
    assert rc == lib.ERR_INVALID and b"bad storage" in L.lbdps_last_error()


def test_missing_library_fails_loudly(lib, monkeypatch):
    # no fallback: without liblbdps.so every entry point raises
    from paper_1303_2653_gb300 import workloads as W
    monkeypatch.setattr(lib, "LIB_PATH", os.path.join(ROOT, "_build", "absent", "liblbdps.so"))
    monkeypatch.setattr(lib, "_LIB", None)
    with pytest.raises(RuntimeError, match="missing"):
        lib.lib()
    with pytest.raises(RuntimeError, match="missing"):
        lib.memory_estimate(W.bubbling2d(nx=16, ny=32, n_particles=10))


def test_product_never_reaches_the_oracle():
    # the package (Python, CUDA, C) neither imports, includes, links nor
    # loads anything of the oracle
    import ast
    pkg = os.path.join(ROOT, "paper_1303_2653_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        mods = [a.name for a in node.names]
                    elif isinstance(node, ast.ImportFrom):
                        mods = [node.module or ""]
                    else:
                        continue
                    assert not any(m.split(".")[0] == "oracle" for m in mods), (path, mods)
                assert "liboracle" not in open(path).read(), path
            elif f.endswith((".cu", ".cuh", ".c", ".h")):
                text = open(path).read()
                assert "lbdps_oracle" not in text and "liboracle" not in text, path
                assert not re.search(r"\bob_[a-z]+\(", text), path


def test_server_reports_a_request_it_cannot_create(lib):
    # without a device, creating the bed of an admitted request fails with
    # LBDPS_ERR_CUDA; the server reports that request as done with the
    # status instead of losing it.  A request larger than the whole budget is
    # refused at submission.
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a GPU")
    L = lib.lib()
    lat, par, prm, keep = _desc(lib)
    s = ctypes.c_void_p()
    assert L.lbdps_server_create(1 << 30, 4, 8, ctypes.byref(s)) == lib.OK
    rid = ctypes.c_uint64(0)
    assert L.lbdps_server_submit(s, ctypes.byref(lat), ctypes.byref(par), ctypes.byref(prm),
                                 10, 0, ctypes.byref(rid)) == lib.OK
    recs, nd = (lib.DoneRec * 4)(), ctypes.c_int(0)
    assert L.lbdps_server_poll(s, 0.0, recs, 4, ctypes.byref(nd)) == lib.OK
    assert nd.value == 1 and recs[0].id == rid.value and recs[0].status == lib.ERR_CUDA
    q, a = ctypes.c_int(-1), ctypes.c_int(-1)
    used = ctypes.c_size_t(1)
    L.lbdps_server_load(s, ctypes.byref(q), ctypes.byref(a), ctypes.byref(used))
    assert (q.value, a.value, used.value) == (0, 0, 0)
    L.lbdps_server_destroy(s)
    small = ctypes.c_void_p()
    assert L.lbdps_server_create(1000, 4, 8, ctypes.byref(small)) == lib.OK
    assert L.lbdps_server_submit(small, ctypes.byref(lat), ctypes.byref(par), ctypes.byref(prm),
                                 10, 0, ctypes.byref(rid)) == lib.ERR_CAPACITY
    assert b"exceeds the HBM budget" in L.lbdps_last_error()
    L.lbdps_server_destroy(small)


def test_binding_constants_match_the_header(lib):
    # every integer constant of include/lbdps.h is in the binding under the
    # same name without the LBDPS_ prefix, with the same value
    text = open(os.path.join(ROOT, "include", "lbdps.h")).read()
    found = 0
    for name, val in re.findall(r"^#define (LBDPS_[A-Z0-9_]+)[ \t]+([^/\n]+)", text, flags=re.M):
        val = val.strip()
        m = re.fullmatch(r"\(?(-?\d+)\)?", val) or re.fullmatch(r"\((\d+)\s*<<\s*(\d+)\)", val)
        if not m:
            continue
        value = int(m.group(1)) << int(m.group(2)) if m.lastindex == 2 else int(m.group(1))
        py = name[len("LBDPS_"):]
        assert hasattr(lib, py), name
        assert getattr(lib, py) == value, (name, getattr(lib, py), value)
        found += 1
    assert found >= 35


def test_binding_structs_match_the_header_layout(lib):
    # offsets and sizes of the ctypes structures equal those a C compiler
    # gives the header's structs (a C program built against include/lbdps.h
    # prints them)
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    structs = {"lbdps_lattice_desc": lib.LatticeDesc, "lbdps_particle_desc": lib.ParticleDesc,
               "lbdps_params": lib.Params, "lbdps_stats_t": lib.Stats, "lbdps_done_t": lib.DoneRec}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbdps.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    scratch = os.path.join(ROOT, "_build", "layout")
    os.makedirs(scratch, exist_ok=True)
    src, exe = os.path.join(scratch, "layout.c"), os.path.join(scratch, "layout")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", exe, src],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    want = {}
    for ln in filter(None, out):
        parts = ln.split()
        want[tuple(parts[:-1])] = int(parts[-1])
    for cname, cls in structs.items():
        assert ctypes.sizeof(cls) == want[(cname, "size")], cname
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == want[(cname, field)], (cname, field)
