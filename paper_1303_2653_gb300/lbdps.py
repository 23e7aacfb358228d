"""Python binding of the C ABI in ``include/lbdps.h`` (argument marshalling only).

Every step of the coupled LB-DPS step runs in the CUDA library
``liblbdps.so``; this module converts Python/NumPy arguments, supplies a
PyTorch CUDA stream and PyTorch's caching allocator to the library, and raises
on non-zero status codes.  There is no fallback: if the library is missing
the import of a bed fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbdps.so")

OK, ERR_INVALID, ERR_OOM, ERR_CAPACITY, ERR_DIVERGED, ERR_DOMAIN, ERR_TIMEOUT, ERR_CUDA = \
    0, -1, -2, -3, -4, -5, -6, -7
WALL, PERIODIC, INLET, OUTLET = 0, 1, 2, 3
STORE_F64, STORE_F32, STORE_F16, STORE_BF16 = 0, 1, 2, 3
UNITS_LATTICE, UNITS_SI = 0, 1

FIELD_RHO, FIELD_U, FIELD_FPG, FIELD_BETA = 1, 2, 4, 8
FIELD_VS, FIELD_NTOT, FIELD_TAU_T, FIELD_UACT, FIELD_EPS_G = 16, 32, 64, 128, 256
VOIDAGE_2D, VOIDAGE_G = 0, 1
FIELD_NAMES = ["rho", "u", "fpg", "beta", "vs", "ntot", "tau_t", "uact", "eps_g"]
VECTOR_FIELDS = {"u", "fpg", "vs", "uact"}
PDIAG_FPRE, PDIAG_FD, PDIAG_BEST, PDIAG_WALL, PDIAG_CELL, PDIAG_ORDER, PDIAG_FC = range(7)
COLLIDE_HARD, COLLIDE_SOFT = 0, 1
CONST_NAMES = ["tau", "nu", "mu", "rho_s", "d", "r", "vp", "mp", "e", "g_eff_x", "g_eff_y",
               "g_eff_z", "fb_x", "fb_y", "fb_z", "u0_x", "u0_y", "u0_z", "cs_smag",
               "kn", "eta", "eta_w", "mu_f", "gamma_t", "inertia"]
KERNEL_CLASSES = ["collide_stream", "drag", "sort", "collide_particles"]

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class LatticeDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("bc", ctypes.c_int * 6),
                ("h", ctypes.c_double), ("dt", ctypes.c_double), ("inlet_u", _dp),
                ("wall_u", (ctypes.c_double * 3) * 6)]


class ParticleDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d_p", ctypes.c_double), ("rho_s", ctypes.c_double),
                ("e", ctypes.c_double), ("pos", _dp), ("vel", _dp),
                ("recirculate", ctypes.c_int), ("collision_model", ctypes.c_int),
                ("dem_kn", ctypes.c_double), ("dem_mu", ctypes.c_double),
                ("dem_gamma_t", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("rho_g", ctypes.c_double), ("mu_g", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("body_accel", ctypes.c_double * 3),
                ("u0", ctypes.c_double * 3), ("cs_smag", ctypes.c_double),
                ("superficial_mode", ctypes.c_int), ("pressure_plus", ctypes.c_int),
                ("storage", ctypes.c_int), ("check_every", ctypes.c_int),
                ("diagnostics", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("gas_momentum", ctypes.c_double * 3),
                ("particle_momentum", ctypes.c_double * 3), ("mean_eps_g", ctypes.c_double),
                ("mean_slip", ctypes.c_double), ("steps", ctypes.c_int64),
                ("health", ctypes.c_int), ("solids_out", ctypes.c_int64)]


class DoneRec(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("steps", ctypes.c_int64),
                ("cells", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("stats", Stats)]


class LbdpsError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str):
        super().__init__(f"{what}: {detail} (status {code})")
        self.code = code


_LIB = None


def lib():
    """Load liblbdps.so (built in-tree by the package build step)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_1303_2653_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "lbdps_create": ([ctypes.POINTER(LatticeDesc), ctypes.POINTER(ParticleDesc),
                              ctypes.POINTER(Params), ctypes.POINTER(vp)], i),
            "lbdps_destroy": ([vp], None),
            "lbdps_step": ([vp, i64], i),
            "lbdps_step_profiled": ([vp, i64, _dp, i, ctypes.POINTER(i)], i),
            "lbdps_step_monitored": ([vp, i64, ctypes.POINTER(Stats)], i),
            "lbdps_sync": ([vp], i),
            "lbdps_fields": ([vp, i, i, _dp, sz], i),
            "lbdps_particles": ([vp, i, _dp, _dp, i64], i),
            "lbdps_set_particles": ([vp, i64, _dp, _dp], i),
            "lbdps_particle_spin": ([vp, i, _dp, i64], i),
            "lbdps_set_particle_spin": ([vp, _dp, i64], i),
            "lbdps_populations": ([vp, _dp, sz], i),
            "lbdps_set_populations": ([vp, _dp, sz], i),
            "lbdps_particle_diag": ([vp, i, _dp, sz], i),
            "lbdps_collide_particles": ([vp, _i64p, i64, _i64p], i),
            "lbdps_stats": ([vp, ctypes.POINTER(Stats)], i),
            "lbdps_health": ([vp, ctypes.POINTER(i)], i),
            "lbdps_constants": ([vp, _dp, i], i),
            "lbdps_shape": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), _i64p, _i64p], i),
            "lbdps_save": ([vp, vp, sz, ctypes.POINTER(sz)], i),
            "lbdps_load": ([vp, vp, sz], i),
            "lbdps_memory_estimate": ([ctypes.POINTER(LatticeDesc), ctypes.POINTER(ParticleDesc),
                                       ctypes.POINTER(Params), ctypes.POINTER(sz)], i),
            "lbdps_record_event": ([vp, vp], i),
            "lbdps_bubbles": ([vp, ctypes.c_double, i, ctypes.POINTER(ctypes.c_int64)], i),
            "lbdps_set_inlet": ([vp, _dp], i),
            "lbdps_check_guards": ([vp, ctypes.POINTER(i)], i),
            "lbdps_server_create": ([sz, i, i, ctypes.POINTER(vp)], i),
            "lbdps_server_submit": ([vp, ctypes.POINTER(LatticeDesc), ctypes.POINTER(ParticleDesc),
                                     ctypes.POINTER(Params), i64, i, ctypes.POINTER(ctypes.c_uint64)], i),
            "lbdps_server_poll": ([vp, ctypes.c_double, ctypes.POINTER(DoneRec), i,
                                   ctypes.POINTER(i)], i),
            "lbdps_server_load": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(sz)], i),
            "lbdps_server_take": ([vp, ctypes.c_uint64, ctypes.POINTER(vp)], i),
            "lbdps_server_destroy": ([vp], None),
            "lbdps_server_set_batching": ([vp, i, i64], i),
            "lbdps_server_batch_info": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                         ctypes.POINTER(i)], i),
            "lbdps_bin_sort_noalloc": ([i, ctypes.POINTER(i), i64, ctypes.POINTER(vp), vp, vp, vp], i),
            "lbdps_strerror": ([i], ctypes.c_char_p),
            "lbdps_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


def _check(code: int, what: str):
    if code != OK:
        detail = lib().lbdps_last_error().decode(errors="replace")
        raise LbdpsError(code, what, detail)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def bin_sort_noalloc(dim: int, n, pos_ptrs, cell_start_ptr: int, order_ptr: int, np_: int,
                     stream_ptr: int = 0):
    """Cell binning on caller-owned device buffers without any device
    allocation (see ``lbdps_bin_sort_noalloc`` in include/lbdps.h).

    ``pos_ptrs`` are device addresses of the FP64 coordinates per axis
    (lattice units), ``cell_start_ptr`` / ``order_ptr`` device addresses of
    the int32 outputs (ncell + 1 and np entries), ``stream_ptr`` a
    cudaStream_t address.  Asynchronous on that stream."""
    nn = (ctypes.c_int * 3)(*(list(int(v) for v in n) + [1] * (3 - len(n))))
    pp = (ctypes.c_void_p * 3)(*([int(p) for p in pos_ptrs] + [None] * (3 - len(pos_ptrs))))
    _check(lib().lbdps_bin_sort_noalloc(int(dim), nn, int(np_), pp, ctypes.c_void_p(cell_start_ptr),
                                        ctypes.c_void_p(order_ptr), ctypes.c_void_p(stream_ptr)),
           "lbdps_bin_sort_noalloc")


def describe(w, storage: Optional[int] = None, diagnostics: bool = False,
             use_graph: bool = True, check_every: int = 0):
    """C descriptions of a workload; returns (lattice, particles, params,
    keepalive arrays).  No allocator and no stream are set."""
    keep = []
    lat = LatticeDesc()
    lat.dim = w.dim
    for a in range(3):
        lat.n[a] = int(w.n[a]) if a < len(w.n) else 1
    for f in range(6):
        lat.bc[f] = int(w.bc[f])
    lat.h, lat.dt = float(w.h), float(w.dt)
    if w.inlet_u is not None:
        iu = np.ascontiguousarray(w.inlet_u, dtype=np.float64)
        keep.append(iu)
        lat.inlet_u = _ptr(iu)
    if w.wall_u is not None:
        for f in range(6):
            for a in range(3):
                lat.wall_u[f][a] = float(w.wall_u[f][a])
    pos = np.ascontiguousarray(w.pos, dtype=np.float64)
    vel = np.ascontiguousarray(w.vel, dtype=np.float64)
    keep += [pos, vel]
    par = ParticleDesc(pos.shape[0], float(w.d_p), float(w.rho_s), float(w.e), _ptr(pos),
                       _ptr(vel), int(w.recirculate), int(getattr(w, "collision_model", 0)),
                       float(getattr(w, "dem_kn", 0.0)), float(getattr(w, "dem_mu", 0.0)),
                       float(getattr(w, "dem_gamma_t", 0.0)))
    prm = Params()
    prm.rho_g, prm.mu_g = float(w.rho_g), float(w.mu_g)
    for a in range(3):
        prm.g[a] = float(w.g[a])
        prm.body_accel[a] = float(w.body_accel[a])
        prm.u0[a] = float(w.u0[a])
    prm.cs_smag = float(w.cs_smag)
    prm.superficial_mode = int(w.superficial_mode)
    prm.pressure_plus = int(w.pressure_plus)
    prm.storage = int(w.storage if storage is None else storage)
    prm.check_every = int(check_every)
    prm.diagnostics = int(bool(diagnostics))
    prm.use_graph = int(bool(use_graph))
    return lat, par, prm, keep


def memory_estimate(w, storage: Optional[int] = None, diagnostics: bool = False) -> int:
    """Exact device bytes of the bed lbdps_create would build."""
    lat, par, prm, keep = describe(w, storage, diagnostics)
    out = ctypes.c_size_t()
    _check(lib().lbdps_memory_estimate(ctypes.byref(lat), ctypes.byref(par), ctypes.byref(prm),
                                       ctypes.byref(out)), "lbdps_memory_estimate")
    return out.value


class Bed:
    """One bed advanced by the CUDA library.

    ``w`` is a :class:`paper_1303_2653_gb300.workloads.Workload` (SI units).
    A dedicated PyTorch CUDA stream carries all work, and device memory comes
    from PyTorch's caching allocator on that stream.
    """

    def __init__(self, w, storage: Optional[int] = None, diagnostics: bool = False,
                 use_graph: bool = True, check_every: int = 0, torch_memory: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self._torch = torch
        self.dim = w.dim
        self.stream = torch.cuda.Stream()
        lat, par, prm, self._keep = describe(w, storage, diagnostics, use_graph, check_every)
        prm.stream = ctypes.c_void_p(self.stream.cuda_stream)
        if torch_memory:
            stream = self.stream
            dev = torch.cuda.current_device()

            def _alloc(nbytes, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
                except Exception:
                    return None

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            prm.alloc = self._alloc_cb
            prm.free = self._free_cb
        handle = ctypes.c_void_p()
        _check(lib().lbdps_create(ctypes.byref(lat), ctypes.byref(par), ctypes.byref(prm),
                                  ctypes.byref(handle)), "lbdps_create")
        self._h = handle
        d, q, nc, npart = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().lbdps_shape(self._h, ctypes.byref(d), ctypes.byref(q), ctypes.byref(nc),
                                 ctypes.byref(npart)), "lbdps_shape")
        self.q, self.ncell, self.np = q.value, nc.value, npart.value
        self.n = tuple(int(w.n[a]) for a in range(w.dim))
        self.storage = prm.storage
        self.diagnostics = bool(diagnostics)

    @classmethod
    def adopt(cls, handle: ctypes.c_void_p, w, diagnostics: bool = False) -> "Bed":
        """Wrap a handle created elsewhere (for example taken from a Server)."""
        self = cls.__new__(cls)
        self._h = handle
        self.dim = w.dim
        self.stream = None
        self._keep = []
        d, q, nc, npart = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().lbdps_shape(self._h, ctypes.byref(d), ctypes.byref(q), ctypes.byref(nc),
                                 ctypes.byref(npart)), "lbdps_shape")
        self.q, self.ncell, self.np = q.value, nc.value, npart.value
        self.n = tuple(int(w.n[a]) for a in range(w.dim))
        self.storage = None
        self.diagnostics = diagnostics
        return self

    # -- life cycle ---------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h and h.value:
            lib().lbdps_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stepping -----------------------------------------------------------
    def step(self, n: int = 1):
        _check(lib().lbdps_step(self._h, int(n)), "lbdps_step")

    def step_profiled(self, n: int = 1) -> Dict[str, float]:
        out = np.zeros(len(KERNEL_CLASSES))
        ncls = ctypes.c_int()
        _check(lib().lbdps_step_profiled(self._h, int(n), _ptr(out), len(out), ctypes.byref(ncls)),
               "lbdps_step_profiled")
        return dict(zip(KERNEL_CLASSES, out.tolist()))

    def sync(self):
        _check(lib().lbdps_sync(self._h), "lbdps_sync")

    # -- data -----------------------------------------------------------------
    def fields(self, mask: int = FIELD_RHO | FIELD_UACT | FIELD_FPG | FIELD_BETA,
               units: int = UNITS_LATTICE) -> Dict[str, np.ndarray]:
        sizes = []
        for bit, name in enumerate(FIELD_NAMES):
            if mask & (1 << bit):
                sizes.append((name, self.ncell * (self.dim if name in VECTOR_FIELDS else 1)))
        total = sum(s for _, s in sizes)
        out = np.empty(max(total, 1))
        _check(lib().lbdps_fields(self._h, int(mask), int(units), _ptr(out), total), "lbdps_fields")
        res, o = {}, 0
        for name, s in sizes:
            arr = out[o:o + s]
            res[name] = arr.reshape(self.ncell, self.dim) if name in VECTOR_FIELDS else arr.copy()
            o += s
        return res

    def particles(self, units: int = UNITS_LATTICE):
        pos = np.empty((max(self.np, 1), self.dim))
        vel = np.empty((max(self.np, 1), self.dim))
        _check(lib().lbdps_particles(self._h, int(units), _ptr(pos), _ptr(vel), self.np),
               "lbdps_particles")
        return pos[: self.np], vel[: self.np]

    def set_particles(self, pos, vel):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        vel = np.ascontiguousarray(vel, dtype=np.float64)
        _check(lib().lbdps_set_particles(self._h, pos.shape[0], _ptr(pos), _ptr(vel)),
               "lbdps_set_particles")

    def spin(self, units: int = UNITS_LATTICE) -> np.ndarray:
        """Particle spins in id order: (N,) in 2D, (N, 3) in 3D."""
        nc = 1 if self.dim == 2 else 3
        out = np.empty(max(self.np, 1) * nc)
        _check(lib().lbdps_particle_spin(self._h, int(units), _ptr(out), self.np * nc),
               "lbdps_particle_spin")
        out = out[: self.np * nc]
        return out if nc == 1 else out.reshape(self.np, 3)

    def set_spin(self, w):
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
        _check(lib().lbdps_set_particle_spin(self._h, _ptr(w), self.np), "lbdps_set_particle_spin")

    def populations(self) -> np.ndarray:
        out = np.empty((self.q, self.ncell))
        _check(lib().lbdps_populations(self._h, _ptr(out), out.size), "lbdps_populations")
        return out

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.q, self.ncell)
        _check(lib().lbdps_set_populations(self._h, _ptr(f), f.size), "lbdps_set_populations")

    def particle_diag(self, which: int) -> np.ndarray:
        vec = which in (PDIAG_FPRE, PDIAG_FD, PDIAG_FC)
        n = self.np * (self.dim if vec else 1)
        out = np.empty(max(n, 1))
        _check(lib().lbdps_particle_diag(self._h, int(which), _ptr(out), n), "lbdps_particle_diag")
        out = out[:n]
        return out.reshape(self.np, self.dim) if vec else out

    def collide_particles(self, record_pairs: bool = True, cap: Optional[int] = None):
        npairs = ctypes.c_int64()
        if not record_pairs:
            _check(lib().lbdps_collide_particles(self._h, None, 0, ctypes.byref(npairs)),
                   "lbdps_collide_particles")
            return None
        cap = int(cap if cap is not None else 8 * max(self.np, 1))
        buf = np.empty((cap, 2), dtype=np.int64)
        _check(lib().lbdps_collide_particles(self._h, buf.ctypes.data_as(_i64p), cap,
                                             ctypes.byref(npairs)), "lbdps_collide_particles")
        return buf[: npairs.value].copy()

    @staticmethod
    def _stats_dict(s) -> dict:
        return {"mass": s.mass, "gas_momentum": np.array(s.gas_momentum[:]),
                "particle_momentum": np.array(s.particle_momentum[:]),
                "mean_eps_g": s.mean_eps_g, "mean_slip": s.mean_slip, "steps": s.steps,
                "health": s.health, "solids_out": s.solids_out}

    def stats(self) -> dict:
        s = Stats()
        _check(lib().lbdps_stats(self._h, ctypes.byref(s)), "lbdps_stats")
        return self._stats_dict(s)

    def step_monitored(self, n: int) -> list:
        """n steps with the statistics after each one (one dict per step)."""
        recs = (Stats * max(int(n), 1))()
        _check(lib().lbdps_step_monitored(self._h, int(n), recs), "lbdps_step_monitored")
        return [self._stats_dict(recs[k]) for k in range(int(n))]

    def bubbles(self, threshold: float = 0.85, voidage: int = 0) -> dict:
        """voidage: VOIDAGE_2D (Eq. 10) or VOIDAGE_G (Eq. 11)."""
        out = (ctypes.c_int64 * 3)()
        _check(lib().lbdps_bubbles(self._h, float(threshold), int(voidage), out), "lbdps_bubbles")
        return {"largest": int(out[0]), "count": int(out[1]), "cells": int(out[2])}

    def check_guards(self) -> int:
        """Number of device buffers written past their end (0 when sound)."""
        n = ctypes.c_int()
        _check(lib().lbdps_check_guards(self._h, ctypes.byref(n)), "lbdps_check_guards")
        return n.value

    def set_inlet(self, inlet_u) -> None:
        u = np.ascontiguousarray(inlet_u, dtype=np.float64)
        _check(lib().lbdps_set_inlet(self._h, _ptr(u)), "lbdps_set_inlet")

    def health(self) -> int:
        hw = ctypes.c_int()
        _check(lib().lbdps_health(self._h, ctypes.byref(hw)), "lbdps_health")
        return hw.value

    def constants(self) -> dict:
        out = np.zeros(len(CONST_NAMES))
        _check(lib().lbdps_constants(self._h, _ptr(out), len(out)), "lbdps_constants")
        return dict(zip(CONST_NAMES, out.tolist()))

    def save(self) -> bytes:
        used = ctypes.c_size_t()
        _check(lib().lbdps_save(self._h, None, 0, ctypes.byref(used)), "lbdps_save")
        buf = ctypes.create_string_buffer(used.value)
        _check(lib().lbdps_save(self._h, buf, used.value, ctypes.byref(used)), "lbdps_save")
        return buf.raw

    def load(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(lib().lbdps_load(self._h, buf, len(data)), "lbdps_load")


class Server:
    """Continuous batching of independent beds (see lbdps_server_* in
    include/lbdps.h).  Beds get their own CUDA streams and device memory from
    cudaMalloc inside the library; the budget bounds their total footprint."""

    def __init__(self, hbm_budget: int, max_active: int = 64, steps_per_tick: int = 16,
                 batching: bool = True, batch_max_cells: int = 0):
        h = ctypes.c_void_p()
        _check(lib().lbdps_server_create(int(hbm_budget), int(max_active), int(steps_per_tick),
                                         ctypes.byref(h)), "lbdps_server_create")
        self._h = h
        _check(lib().lbdps_server_set_batching(self._h, int(bool(batching)), int(batch_max_cells)),
               "lbdps_server_set_batching")
        self._workloads = {}
        self._callbacks = []

    def submit(self, w, steps: int, storage: Optional[int] = None, keep: bool = False,
               alloc=None, free=None, diagnostics: bool = False) -> int:
        """Queue a bed for `steps` steps.  `alloc(nbytes) -> int|None` and
        `free(ptr)` optionally replace cudaMalloc/cudaFree for this bed;
        `diagnostics` keeps the node diagnostics (needed for the mean slip
        of the completion record)."""
        lat, par, prm, keepalive = describe(w, storage, diagnostics)
        if alloc is not None:
            cb_a = ALLOC_FN(lambda n, ctx: alloc(n))
            cb_f = FREE_FN(lambda ptr, ctx: free(ptr) if free else None)
            prm.alloc, prm.free = cb_a, cb_f
            self._callbacks.append((cb_a, cb_f))
        rid = ctypes.c_uint64()
        _check(lib().lbdps_server_submit(self._h, ctypes.byref(lat), ctypes.byref(par),
                                         ctypes.byref(prm), int(steps), int(bool(keep)),
                                         ctypes.byref(rid)), "lbdps_server_submit")
        if keep:
            self._workloads[rid.value] = w
        return rid.value

    def poll(self, wait_s: float = 0.0, cap: int = 256):
        buf = (DoneRec * cap)()
        n = ctypes.c_int()
        _check(lib().lbdps_server_poll(self._h, float(wait_s), buf, cap, ctypes.byref(n)),
               "lbdps_server_poll")
        out = []
        for r in buf[: n.value]:
            out.append({"id": r.id, "status": r.status, "steps": r.steps, "cells": r.cells,
                        "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done,
                        "mass": r.stats.mass, "mean_eps_g": r.stats.mean_eps_g,
                        "mean_slip": r.stats.mean_slip, "health": r.stats.health})
        return out

    def load(self):
        q, a, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(lib().lbdps_server_load(self._h, ctypes.byref(q), ctypes.byref(a), ctypes.byref(u)),
               "lbdps_server_load")
        return q.value, a.value, u.value

    def batch_info(self):
        """(ticks launched, graph captures, current members) of the batch."""
        t, c, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().lbdps_server_batch_info(self._h, ctypes.byref(t), ctypes.byref(c),
                                             ctypes.byref(m)), "lbdps_server_batch_info")
        return t.value, c.value, m.value

    def take(self, req_id: int) -> Bed:
        h = ctypes.c_void_p()
        _check(lib().lbdps_server_take(self._h, ctypes.c_uint64(req_id), ctypes.byref(h)),
               "lbdps_server_take")
        return Bed.adopt(h, self._workloads.pop(req_id))

    def close(self):
        h = getattr(self, "_h", None)
        if h and h.value:
            lib().lbdps_server_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
