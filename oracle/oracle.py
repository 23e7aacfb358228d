"""ctypes front end of the CPU oracle (test infrastructure only).

The oracle is a plain FP64 C restatement of one coupled LB-DPS step
(``lbdps_oracle.c``).  Only tests, the package smoke check and the benchmark's
CPU-baseline leg use it.  It takes any object with the workload attributes
(``dim, n, bc, h, dt, d_p, rho_s, e, pos, vel, rho_g, mu_g, g, body_accel,
u0, inlet_u, wall_u, cs_smag, superficial_mode, pressure_plus``); it does not
import the CUDA package.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

F_RHO, F_U, F_UACT, F_VS, F_EPS_S, F_EPS_G, F_OMEGA, F_BETA, F_FPG, F_GRADP, F_TAU_T, \
    F_NTOT, F_SUM_PRE, F_SUM_ABS_PRE, F_EPS_2D = range(15)
VECTOR_FIELDS = {F_U, F_UACT, F_VS, F_FPG, F_GRADP, F_SUM_PRE, F_SUM_ABS_PRE}
P_FPRE, P_FD, P_CELL, P_BEST, P_WALL, P_FC = range(6)
CONST_NAMES = ["tau", "nu", "mu", "rho_s", "d", "r", "vp", "mp", "e", "g_eff_x", "g_eff_y",
               "g_eff_z", "fb_x", "fb_y", "fb_z", "u0_x", "u0_y", "u0_z", "cs_smag",
               "kn", "eta", "eta_w", "mu_f", "gamma_t", "inertia"]


class Setup(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("bc", ctypes.c_int * 6),
        ("h", ctypes.c_double), ("dt", ctypes.c_double),
        ("inlet_u", ctypes.POINTER(ctypes.c_double)),
        ("wall_u", (ctypes.c_double * 3) * 6),
        ("np", ctypes.c_int64), ("d_p", ctypes.c_double), ("rho_s", ctypes.c_double),
        ("e", ctypes.c_double),
        ("pos", ctypes.POINTER(ctypes.c_double)), ("vel", ctypes.POINTER(ctypes.c_double)),
        ("rho_g", ctypes.c_double), ("mu_g", ctypes.c_double),
        ("g", ctypes.c_double * 3), ("body_accel", ctypes.c_double * 3),
        ("u0", ctypes.c_double * 3), ("cs_smag", ctypes.c_double),
        ("superficial_mode", ctypes.c_int), ("pressure_plus", ctypes.c_int),
        ("recirculate", ctypes.c_int), ("collision_model", ctypes.c_int),
        ("dem_kn", ctypes.c_double), ("dem_mu", ctypes.c_double),
        ("dem_gamma_t", ctypes.c_double), ("collision_rule", ctypes.c_int),
    ]


def lib():
    global _LIB
    if _LIB is None:
        # LBDPS_ORACLE_LIB names another build of the oracle source: the
        # mutation check of the pins loads its planted-mistake libraries so
        path = os.environ.get("LBDPS_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        d = ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        L.ob_create.argtypes = [ctypes.POINTER(Setup)]
        L.ob_create.restype = vp
        L.ob_destroy.argtypes = [vp]
        L.ob_step.argtypes = [vp]
        L.ob_run.argtypes = [vp, ctypes.c_int64]
        L.ob_collide_particles.argtypes = [vp]
        for name in ("ob_dim", "ob_nq"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = ctypes.c_int
        for name in ("ob_ncell", "ob_np", "ob_npairs", "ob_solids_out"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = ctypes.c_int64
        L.ob_constants.argtypes = [vp, dp]
        L.ob_set_inlet.argtypes = [vp, dp]
        L.ob_bubbles.argtypes = [vp, d, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
        L.ob_units_flat.argtypes = [ctypes.POINTER(Setup), dp]
        L.ob_get_populations.argtypes = [vp, dp]
        L.ob_set_populations.argtypes = [vp, dp]
        L.ob_get_particles.argtypes = [vp, dp, dp]
        L.ob_set_particles.argtypes = [vp, ctypes.c_int64, dp, dp]
        L.ob_set_particles.restype = ctypes.c_int
        L.ob_get_sorted.argtypes = [vp, i64p, i64p]
        L.ob_get_spin.argtypes = [vp, dp]
        L.ob_set_spin.argtypes = [vp, dp]
        L.ob_get_field.argtypes = [vp, ctypes.c_int, dp]
        L.ob_get_field.restype = ctypes.c_int
        L.ob_get_particle_diag.argtypes = [vp, ctypes.c_int, dp]
        L.ob_get_particle_diag.restype = ctypes.c_int
        L.ob_get_pairs.argtypes = [vp, i64p, ctypes.c_int64]
        L.ob_get_pairs.restype = ctypes.c_int64
        L.ob_stats.argtypes = [vp, dp]
        for name in ("ob_gamma",):
            getattr(L, name).argtypes = [d, d]
            getattr(L, name).restype = d
        for name in ("ob_eps3d", "ob_omega"):
            getattr(L, name).argtypes = [d]
            getattr(L, name).restype = d
        L.ob_reynolds.argtypes = [d, d, d, d, d]
        L.ob_reynolds.restype = d
        L.ob_beta.argtypes = [d, d, d, d, d]
        L.ob_beta.restype = d
        L.ob_binary_collision.argtypes = [ctypes.c_int, d, d, d, dp, dp, dp, dp]
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def make_setup(w):
    """Fill a Setup from a workload-like object; returns (setup, keepalive)."""
    s = Setup()
    s.dim = w.dim
    for a in range(3):
        s.n[a] = int(w.n[a]) if a < len(w.n) else 1
    for f in range(6):
        s.bc[f] = int(w.bc[f])
    s.h, s.dt = float(w.h), float(w.dt)
    keep = []
    if getattr(w, "inlet_u", None) is not None:
        iu = np.ascontiguousarray(w.inlet_u, dtype=np.float64)
        keep.append(iu)
        s.inlet_u = _dp(iu)
    wall_u = getattr(w, "wall_u", None)
    if wall_u is not None:
        for f in range(6):
            for a in range(3):
                s.wall_u[f][a] = float(wall_u[f][a])
    pos = np.ascontiguousarray(w.pos, dtype=np.float64)
    vel = np.ascontiguousarray(w.vel, dtype=np.float64)
    keep += [pos, vel]
    s.np = pos.shape[0]
    s.pos, s.vel = _dp(pos), _dp(vel)
    s.d_p, s.rho_s, s.e = float(w.d_p), float(w.rho_s), float(w.e)
    s.rho_g, s.mu_g = float(w.rho_g), float(w.mu_g)
    for a in range(3):
        s.g[a] = float(w.g[a])
        s.body_accel[a] = float(w.body_accel[a])
        s.u0[a] = float(w.u0[a])
    s.cs_smag = float(w.cs_smag)
    s.superficial_mode = int(w.superficial_mode)
    s.pressure_plus = int(w.pressure_plus)
    s.recirculate = int(getattr(w, "recirculate", False))
    s.collision_model = int(getattr(w, "collision_model", 0))
    s.dem_kn = float(getattr(w, "dem_kn", 0.0))
    s.dem_mu = float(getattr(w, "dem_mu", 0.0))
    s.dem_gamma_t = float(getattr(w, "dem_gamma_t", 0.0))
    s.collision_rule = int(getattr(w, "collision_rule", 0))
    return s, keep


def units(w) -> dict:
    s, keep = make_setup(w)
    out = np.zeros(len(CONST_NAMES))
    lib().ob_units_flat(ctypes.byref(s), _dp(out))
    return dict(zip(CONST_NAMES, out))


def gamma(eps_s, tau):
    return lib().ob_gamma(eps_s, tau)


def eps3d(eps_2d):
    return lib().ob_eps3d(eps_2d)


def omega(eps_g):
    return lib().ob_omega(eps_g)


def beta(eps_g, slip, rho_g, mu, d):
    return lib().ob_beta(eps_g, slip, rho_g, mu, d)


def binary_collision(dim, m1, m2, e, p1, p2, v1, v2):
    p1 = np.array(p1, dtype=np.float64); p2 = np.array(p2, dtype=np.float64)
    v1 = np.array(v1, dtype=np.float64); v2 = np.array(v2, dtype=np.float64)
    lib().ob_binary_collision(dim, m1, m2, e, _dp(p1), _dp(p2), _dp(v1), _dp(v2))
    return v1, v2


class OracleBed:
    """One bed stepped by the FP64 oracle."""

    def __init__(self, w):
        s, keep = make_setup(w)
        self._h = lib().ob_create(ctypes.byref(s))
        if not self._h:
            raise ValueError("oracle rejected the bed description")
        self.dim = lib().ob_dim(self._h)
        self.nq = lib().ob_nq(self._h)
        self.ncell = lib().ob_ncell(self._h)
        self.n = tuple(int(w.n[a]) for a in range(self.dim))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _LIB is not None:
            _LIB.ob_destroy(h)
            self._h = None

    @property
    def np(self):
        return lib().ob_np(self._h)

    def step(self, n: int = 1):
        lib().ob_run(self._h, int(n))

    def collide_particles(self):
        """Sort, detect and resolve hard-sphere contacts on the current state."""
        lib().ob_collide_particles(self._h)

    def constants(self) -> dict:
        out = np.zeros(len(CONST_NAMES))
        lib().ob_constants(self._h, _dp(out))
        return dict(zip(CONST_NAMES, out))

    def populations(self) -> np.ndarray:
        out = np.empty((self.nq, self.ncell))
        lib().ob_get_populations(self._h, _dp(out))
        return out

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.nq, self.ncell)
        lib().ob_set_populations(self._h, _dp(f))

    def particles(self):
        n = self.np
        P = np.empty((n, self.dim)); v = np.empty((n, self.dim))
        lib().ob_get_particles(self._h, _dp(P), _dp(v))
        return P, v

    def set_particles(self, P, v):
        P = np.ascontiguousarray(P, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        if lib().ob_set_particles(self._h, P.shape[0], _dp(P), _dp(v)) != 0:
            raise MemoryError("oracle particle allocation failed")

    def spin(self) -> np.ndarray:
        """Angular velocities in id order (lattice units): (N,) in 2D (the z
        component), (N, 3) in 3D."""
        nc = 1 if self.dim == 2 else 3
        out = np.empty(max(self.np, 1) * nc)
        lib().ob_get_spin(self._h, _dp(out))
        out = out[: self.np * nc]
        return out if nc == 1 else out.reshape(self.np, 3)

    def set_spin(self, w):
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
        lib().ob_set_spin(self._h, _dp(w))

    def sorted_ids(self):
        ids = np.empty(max(self.np, 1), dtype=np.int64)
        cs = np.empty(self.ncell + 1, dtype=np.int64)
        lib().ob_get_sorted(self._h, _i64p(ids), _i64p(cs))
        return ids[: self.np], cs

    def field(self, which: int) -> np.ndarray:
        vec = which in VECTOR_FIELDS
        out = np.empty(self.ncell * (self.dim if vec else 1))
        if lib().ob_get_field(self._h, which, _dp(out)) != 0:
            raise ValueError(which)
        return out.reshape(self.ncell, self.dim) if vec else out

    def particle_diag(self, which: int) -> np.ndarray:
        vec = which in (P_FPRE, P_FD, P_FC)
        out = np.empty(max(self.np, 1) * (self.dim if vec else 1))
        lib().ob_get_particle_diag(self._h, which, _dp(out))
        out = out[: self.np * (self.dim if vec else 1)]
        return out.reshape(self.np, self.dim) if vec else out

    def pairs(self) -> np.ndarray:
        n = lib().ob_npairs(self._h)
        out = np.empty((max(n, 1), 2), dtype=np.int64)
        lib().ob_get_pairs(self._h, _i64p(out), n)
        return out[:n]

    def set_inlet(self, inlet_u):
        u = np.ascontiguousarray(inlet_u, dtype=np.float64)
        lib().ob_set_inlet(self._h, _dp(u))

    def bubbles(self, threshold: float = 0.85, voidage: int = 0) -> dict:
        out = np.zeros(3, dtype=np.int64)
        lib().ob_bubbles(self._h, float(threshold), int(voidage), _i64p(out))
        return {"largest": int(out[0]), "count": int(out[1]), "cells": int(out[2])}

    def stats(self) -> dict:
        out = np.zeros(9)
        lib().ob_stats(self._h, _dp(out))
        return {"solids_out": int(lib().ob_solids_out(self._h)),
                "mass": out[0], "gas_momentum": out[1:4], "particle_momentum": out[4:7],
                "mean_eps_g": out[7], "mean_slip": out[8]}
