"""Seeded synthetic workloads for the LB-DPS coupled step.

This module only builds inputs: lattice shape, boundary types, SI physical
parameters, and particle positions/velocities drawn by the C generator in
``csrc/workloads.c`` (splitmix64 stream, random sequential addition,
Box-Muller Maxwellian).  It contains none of the method's arithmetic; the
conversion to lattice units happens separately inside the GPU library and
inside the CPU oracle.

Workload shapes follow the paper's two test problems (Tables 1 and 2, §3.1
and §3.2): a bubbling bed with a central jet and a periodic riser section,
plus a D3Q19 riser and small closed-form flows used by tests.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
from typing import Optional

import numpy as np

WALL, PERIODIC, INLET, OUTLET = 0, 1, 2, 3
STORE_F64, STORE_F32, STORE_F16, STORE_BF16 = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "libworkloads.so")
        if not os.path.exists(path):
            from . import build as _build
            _build.build_workloads()
        lib = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        lib.wl_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64, d]
        lib.wl_uniform.restype = None
        lib.wl_maxwellian.argtypes = [ctypes.c_int, ctypes.c_int64, d, ctypes.c_double,
                                      ctypes.c_uint64, d]
        lib.wl_maxwellian.restype = None
        lib.wl_rsa.argtypes = [ctypes.c_int, d, d, d, ctypes.POINTER(ctypes.c_int),
                               ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                               ctypes.c_int64, d]
        lib.wl_rsa.restype = ctypes.c_int64
        _LIB = lib
    return _LIB


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def uniform_stream(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _lib().wl_uniform(ctypes.c_uint64(seed), n, _dptr(out))
    return out


def maxwellian(dim: int, n: int, mean, sigma: float, seed: int) -> np.ndarray:
    out = np.empty(n * dim, dtype=np.float64)
    m = np.zeros(3, dtype=np.float64)
    m[:dim] = mean[:dim]
    _lib().wl_maxwellian(dim, n, _dptr(m), float(sigma), ctypes.c_uint64(seed), _dptr(out))
    return out.reshape(n, dim)


def rsa(dim: int, box, lo, hi, periodic, sep: float, n: int, seed: int,
        max_attempts: Optional[int] = None) -> np.ndarray:
    """Non-overlapping centres (pairwise distance >= sep) in [lo, hi]."""
    b = np.zeros(3); b[:dim] = box[:dim]
    l = np.zeros(3); l[:dim] = lo[:dim]
    h = np.zeros(3); h[:dim] = hi[:dim]
    per = (ctypes.c_int * 3)(*[int(bool(p)) for p in list(periodic[:dim]) + [0] * (3 - dim)])
    out = np.empty(max(n, 1) * dim, dtype=np.float64)
    if max_attempts is None:
        max_attempts = 200 * n + 1000
    got = _lib().wl_rsa(dim, _dptr(b), _dptr(l), _dptr(h), per, float(sep), n,
                        ctypes.c_uint64(seed), int(max_attempts), _dptr(out))
    if got != n:
        raise RuntimeError(f"random sequential addition placed {got} of {n} centres")
    return out[: n * dim].reshape(n, dim).copy()


@dataclasses.dataclass
class Workload:
    """One bed: lattice, particles and physical parameters, all in SI units."""
    name: str
    dim: int
    n: tuple                      # cells per axis (nx, ny[, nz]); last axis is vertical
    bc: tuple                     # per face: x-, x+, y-, y+, z-, z+
    h: float                      # cell size (m)
    dt: float                     # time step (s)
    d_p: float                    # particle diameter (m)
    rho_s: float                  # solid density (kg/m^3)
    e: float                      # restitution coefficient
    pos: np.ndarray               # (N, dim) particle centres (m)
    vel: np.ndarray               # (N, dim) particle velocities (m/s)
    rho_g: float                  # gas density (kg/m^3)
    mu_g: float                   # gas viscosity (Pa s)
    g: tuple = (0.0, 0.0, 0.0)    # gravity (m/s^2)
    body_accel: tuple = (0.0, 0.0, 0.0)   # gas body acceleration (m/s^2)
    u0: tuple = (0.0, 0.0, 0.0)   # initial gas velocity (m/s)
    inlet_u: Optional[np.ndarray] = None  # (cells of the inlet face, dim) m/s
    wall_u: Optional[np.ndarray] = None   # (6, 3) tangential wall velocity (m/s)
    cs_smag: float = 0.0
    superficial_mode: int = 0
    pressure_plus: int = 0
    recirculate: bool = False     # outlet -> inlet re-injection of particles
    collision_model: int = 0      # 0: time-driven hard spheres, 1: soft spheres
    dem_kn: float = 0.0           # soft-sphere normal stiffness (N/m)
    dem_mu: float = 0.0           # soft-sphere Coulomb friction coefficient (0 = none)
    dem_gamma_t: float = 0.0      # soft-sphere tangential damping (kg/s)
    storage: int = STORE_F32
    steps: int = 1
    seed: int = 0

    @property
    def n_particles(self) -> int:
        return int(self.pos.shape[0])

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def _bc(dim, x, y, z=(WALL, WALL)):
    return tuple(list(x) + list(y) + (list(z) if dim == 3 else [PERIODIC, PERIODIC]))


SEED_BASE = 1303000


def bubbling2d(nx=64, ny=128, n_particles=2000, seed=SEED_BASE + 0, storage=STORE_F64,
               steps=500, cs_smag=0.0, jet_cells=4, jet_factor=5.0, u_mf=0.1885,
               dt=1.0e-4, bed_fraction=0.4) -> Workload:
    """Single-jet bubbling bed in the shape of the paper's §3.1 case (Table 1).

    Cell size 2 mm; 0.5 mm, 2500 kg/m^3 particles placed by RSA in the lower
    ``bed_fraction`` of the bed; walls at the sides, a velocity inlet at the
    bottom (u_mf everywhere, ``jet_factor`` x u_mf on the central ``jet_cells``
    cells) and a pressure outlet at the top.
    """
    h = 2.0e-3
    d_p = 0.5e-3
    r = 0.5 * d_p
    W, H = nx * h, ny * h
    pos = rsa(2, (W, H), (r, r), (W - r, bed_fraction * H), (0, 0), d_p * (1 + 1e-9),
              n_particles, seed)
    vel = np.zeros_like(pos)
    inlet = np.zeros((nx, 2))
    inlet[:, 1] = u_mf
    j0 = nx // 2 - jet_cells // 2
    inlet[j0:j0 + jet_cells, 1] = jet_factor * u_mf
    return Workload(
        name=f"bubbling2d-{nx}x{ny}-N{n_particles}", dim=2, n=(nx, ny),
        bc=(WALL, WALL, INLET, OUTLET, PERIODIC, PERIODIC), h=h, dt=dt, d_p=d_p,
        rho_s=2500.0, e=0.9, pos=pos, vel=vel, rho_g=1.2, mu_g=1.8e-5,
        g=(0.0, -9.81, 0.0), u0=(0.0, u_mf, 0.0), inlet_u=inlet, cs_smag=cs_smag,
        storage=storage, steps=steps, seed=seed)


def bubbling_table1(nx=25, ny=100, n_particles=15000, seed=SEED_BASE + 6, storage=STORE_F32,
                    steps=26000, cs_smag=0.0, jet_cells=3, v_mf=0.0025, v_inj=0.8,
                    bed_rows=45) -> Workload:
    """The single-orifice bubbling bed of the paper's §3.1 (Table 1):
    0.00675 m x 0.027 m at h = 2.7e-4 m (25 x 100 cells), dt = 1.35e-6 s,
    15,000 particles of 54 um and 930 kg/m^3 placed at rest by random
    sequential addition in the lower ``bed_rows`` rows (2D area fraction 0.42
    at 45 rows), gas 1.1795 kg/m^3, 1.8872e-5 Pa s, a bottom inlet at the
    minimum fluidization velocity 0.0025 m/s with the central ``jet_cells``
    cells (the 0.00081 m orifice) injecting at 0.8 m/s, a pressure outlet at
    the top and walls at the sides.  The pulse length (0.006 s in §3.1) is
    applied by the caller with lbdps_set_inlet (``background_inlet``)."""
    h, dt = 2.7e-4, 1.35e-6
    d_p = 54e-6
    r = 0.5 * d_p
    W = nx * h
    pos = rsa(2, (W, ny * h), (r, r), (W - r, bed_rows * h), (0, 0), d_p * (1 + 1e-9),
              n_particles, seed)
    vel = np.zeros_like(pos)
    inlet = np.zeros((nx, 2))
    inlet[:, 1] = v_mf
    j0 = nx // 2 - jet_cells // 2
    inlet[j0:j0 + jet_cells, 1] = v_inj
    return Workload(
        name=f"bubbling-table1-{nx}x{ny}-N{n_particles}", dim=2, n=(nx, ny),
        bc=(WALL, WALL, INLET, OUTLET, PERIODIC, PERIODIC), h=h, dt=dt, d_p=d_p,
        rho_s=930.0, e=0.9, pos=pos, vel=vel, rho_g=1.1795, mu_g=1.8872e-5,
        g=(0.0, -9.81, 0.0), u0=(0.0, v_mf, 0.0), inlet_u=inlet, cs_smag=cs_smag,
        storage=storage, steps=steps, seed=seed)


def dem_stiffness(w: Workload, contact_steps: float = 20.0) -> float:
    """Normal stiffness k_n (N/m) that makes an undamped pair contact last
    ``contact_steps`` time steps: half a period pi sqrt(m_eff / k_n) of the
    spring with the reduced mass m_eff = m_p / 2."""
    m_p = w.rho_s * math.pi * w.d_p ** 3 / 6.0
    t_c = contact_steps * w.dt
    return 0.5 * m_p * (math.pi / t_c) ** 2


def soft_spheres(w: Workload, contact_steps: float = 20.0, e: Optional[float] = None) -> Workload:
    """The same bed with the soft-sphere contact model in place of the
    time-driven hard spheres."""
    w2 = w.with_(collision_model=1, name=w.name + "-dem")
    if e is not None:
        w2 = w2.with_(e=e)
    return w2.with_(dem_kn=dem_stiffness(w2, contact_steps))


def with_friction(w: Workload, mu: float = 0.5, gamma_frac: float = 0.05) -> Workload:
    """The soft-sphere bed with friction: Coulomb coefficient ``mu`` and the
    tangential damping ``gamma_frac`` m_p / dt (a sliding pair's slip then
    relaxes by 7 gamma_frac per step)."""
    m_p = w.rho_s * math.pi * w.d_p ** 3 / 6.0
    return w.with_(dem_mu=mu, dem_gamma_t=gamma_frac * m_p / w.dt, name=w.name + "-fric")


def packed_bed(dim=2, n=(32, 64), fill_rows=None, gap=0.9, n_particles=None,
               seed=SEED_BASE + 7, storage=STORE_F64, contact_steps=20.0, e=0.7,
               sigma_v=0.05, cs_smag=0.0) -> Workload:
    """A dense soft-sphere bed of Table 1 particles (54 um, 930 kg/m^3, h =
    2.7e-4 m, dt = 1.35e-6 s) whose centres are only ``gap`` d_p apart at
    least, so that many pairs start in contact: random sequential addition in
    the lower ``fill_rows`` rows of a closed box (walls on every face), gas at
    rest, gravity, Maxwellian velocities of ``sigma_v`` m/s."""
    h, dt, d_p = 2.7e-4, 1.35e-6, 54e-6
    r = 0.5 * d_p
    n = tuple(n)
    if fill_rows is None:
        fill_rows = n[-1] // 2
    lo = [r] * dim
    hi = [n[a] * h - r for a in range(dim)]
    hi[-1] = fill_rows * h
    box = [n[a] * h for a in range(dim)]
    if n_particles is None:
        # about 0.35 of the filled area (2D) or volume (3D) in particles
        if dim == 2:
            n_particles = int(0.35 * box[0] * fill_rows * h / (math.pi * r * r))
        else:
            n_particles = int(0.35 * box[0] * box[1] * fill_rows * h / (math.pi * d_p ** 3 / 6))
    pos = rsa(dim, box, lo, hi, (0, 0, 0), gap * d_p, n_particles, seed)
    vel = maxwellian(dim, n_particles, (0.0,) * dim, sigma_v, seed ^ 0x5DEECE66D)
    bc = _bc(dim, (WALL, WALL), (WALL, WALL), (WALL, WALL))
    g = (0.0, -9.81, 0.0) if dim == 2 else (0.0, 0.0, -9.81)
    w = Workload(
        name=f"packed{dim}d-{'x'.join(map(str, n))}-N{n_particles}", dim=dim, n=n, bc=bc, h=h,
        dt=dt, d_p=d_p, rho_s=930.0, e=e, pos=pos, vel=vel, rho_g=1.1795, mu_g=1.8872e-5, g=g,
        storage=storage, seed=seed, collision_model=1, cs_smag=cs_smag)
    return w.with_(dem_kn=dem_stiffness(w, contact_steps))


def background_inlet(w: Workload) -> np.ndarray:
    """The inlet of a bubbling bed with the jet switched off: every inlet cell
    at the background (minimum fluidization) velocity of its edge cells."""
    u = np.array(w.inlet_u, dtype=np.float64)
    u[:, :] = u[0, :]
    return u


def riser2d(nx=256, ny=2048, n_particles=200000, seed=SEED_BASE + 1, storage=STORE_F32,
            steps=10000, cs_smag=0.0, solid_fraction=0.05, u_gas=1.5, u_lat=0.0338,
            sigma_v=0.1, h=None) -> Workload:
    """Periodic riser section in the shape of the paper's §3.2 case (Table 2).

    54 um, 930 kg/m^3 particles at a mean 2D area fraction ``solid_fraction``
    (the cell size h follows from it), Maxwellian velocities of standard
    deviation ``sigma_v`` per component, gas initially at ``u_gas`` upward,
    time step from the lattice inlet velocity of Table 2, walls at the sides,
    periodic vertically, and an upward gas body acceleration that carries the
    particles' effective weight.  With ``h`` given the cell size is fixed and
    the solid fraction follows from ``n_particles``.
    """
    d_p = 54e-6
    r = 0.5 * d_p
    rho_s, rho_g, mu_g, g = 930.0, 1.1795, 1.8872e-5, 9.81
    if h is None:   # the cell size that gives the requested mean solid fraction
        h = math.sqrt(n_particles * math.pi * r * r / (nx * ny * solid_fraction))
    dt = u_lat * h / u_gas
    W, H = nx * h, ny * h
    pos = rsa(2, (W, H), (r, 0.0), (W - r, H), (0, 1), d_p * (1 + 1e-9), n_particles, seed)
    vel = maxwellian(2, n_particles, (0.0, 0.0), sigma_v, seed ^ 0x5DEECE66D)
    v_p = math.pi * d_p ** 3 / 6.0
    a_body = n_particles * v_p * (rho_s - rho_g) * g / (rho_g * nx * ny * h ** 3)
    return Workload(
        name=f"riser2d-{nx}x{ny}-N{n_particles}", dim=2, n=(nx, ny),
        bc=(WALL, WALL, PERIODIC, PERIODIC, PERIODIC, PERIODIC), h=h, dt=dt, d_p=d_p,
        rho_s=rho_s, e=0.9, pos=pos, vel=vel, rho_g=rho_g, mu_g=mu_g,
        g=(0.0, -g, 0.0), body_accel=(0.0, a_body, 0.0), u0=(0.0, u_gas, 0.0),
        cs_smag=cs_smag, storage=storage, steps=steps, seed=seed)


def cfb_riser2d(nx=60, ny=720, n_particles=123921, seed=SEED_BASE + 5, storage=STORE_F32,
                steps=20000, cs_smag=0.1, h=2.7e-4, u_in=1.52, u_lat=0.0338) -> Workload:
    """The riser of a circulating fluidized bed as in the paper's §3.2 (Table 2):
    0.0162 m x 0.194 m at h = 2.7e-4 m (60 x 720 cells), 123,921 particles of
    54 um and 930 kg/m^3 placed uniformly at rest (solids fraction 0.09),
    gas 1.1795 kg/m^3, 1.8872e-5 Pa s entering at the bottom at 1.52 m/s
    (0.0338 in lattice units, which sets dt = 6.0e-6 s), a pressure outlet at
    the top, walls at the sides, gravity, and the solids loop closed: a
    particle leaving through the outlet re-enters through the inlet.  The
    Smagorinsky constant is a parameter (the paper prints none; tau is
    0.5040).  Smaller lattices keep h and the solids fraction."""
    d_p = 54e-6
    r = 0.5 * d_p
    rho_s, rho_g, mu_g, g = 930.0, 1.1795, 1.8872e-5, 9.81
    dt = u_lat * h / u_in
    W, H = nx * h, ny * h
    pos = rsa(2, (W, H), (r, r), (W - r, H - r), (0, 0), d_p * (1 + 1e-9), n_particles, seed)
    vel = np.zeros_like(pos)
    inlet = np.zeros((nx, 2))
    inlet[:, 1] = u_in
    return Workload(
        name=f"cfbriser2d-{nx}x{ny}-N{n_particles}", dim=2, n=(nx, ny),
        bc=(WALL, WALL, INLET, OUTLET, PERIODIC, PERIODIC), h=h, dt=dt, d_p=d_p,
        rho_s=rho_s, e=0.9, pos=pos, vel=vel, rho_g=rho_g, mu_g=mu_g,
        g=(0.0, -g, 0.0), u0=(0.0, u_in, 0.0), inlet_u=inlet, cs_smag=cs_smag,
        recirculate=True, storage=storage, steps=steps, seed=seed)


def riser3d(nx=256, ny=256, nz=1024, n_particles=4000000, seed=SEED_BASE + 3,
            storage=STORE_F32, steps=2000, cs_smag=0.0, solid_fraction=0.03,
            u_gas=1.5, u_lat=0.0338, sigma_v=0.1) -> Workload:
    """D3Q19 riser: walls in x and y, periodic in z (vertical), volume fraction
    ``solid_fraction`` of 54 um spheres; otherwise as :func:`riser2d`."""
    d_p = 54e-6
    r = 0.5 * d_p
    rho_s, rho_g, mu_g, g = 930.0, 1.1795, 1.8872e-5, 9.81
    v_p = math.pi * d_p ** 3 / 6.0
    h = (n_particles * v_p / (nx * ny * nz * solid_fraction)) ** (1.0 / 3.0)
    dt = u_lat * h / u_gas
    box = (nx * h, ny * h, nz * h)
    pos = rsa(3, box, (r, r, 0.0), (box[0] - r, box[1] - r, box[2]), (0, 0, 1),
              d_p * (1 + 1e-9), n_particles, seed)
    vel = maxwellian(3, n_particles, (0.0, 0.0, 0.0), sigma_v, seed ^ 0x5DEECE66D)
    a_body = n_particles * v_p * (rho_s - rho_g) * g / (rho_g * nx * ny * nz * h ** 3)
    return Workload(
        name=f"riser3d-{nx}x{ny}x{nz}-N{n_particles}", dim=3, n=(nx, ny, nz),
        bc=(WALL, WALL, WALL, WALL, PERIODIC, PERIODIC), h=h, dt=dt, d_p=d_p,
        rho_s=rho_s, e=0.9, pos=pos, vel=vel, rho_g=rho_g, mu_g=mu_g,
        g=(0.0, 0.0, -g), body_accel=(0.0, 0.0, a_body), u0=(0.0, 0.0, u_gas),
        cs_smag=cs_smag, storage=storage, steps=steps, seed=seed)


def channel2d(nx=16, ny=4, h=1.0e-3, dt=1.0e-3, nu=1.0e-4, body_accel=0.0,
              top_wall_u=0.0, storage=STORE_F64, bc_y=PERIODIC, cs_smag=0.0) -> Workload:
    """Particle-free channel for closed-form flows: walls at x-/x+, periodic
    in y.  ``body_accel`` drives Poiseuille flow along +y; ``top_wall_u``
    moves the x+ wall along +y (Couette).  Gas density 1, viscosity nu."""
    wall_u = np.zeros((6, 3))
    wall_u[1, 1] = top_wall_u
    return Workload(
        name=f"channel2d-{nx}x{ny}", dim=2, n=(nx, ny),
        bc=(WALL, WALL, bc_y, bc_y, PERIODIC, PERIODIC), h=h, dt=dt, d_p=0.1 * h,
        rho_s=1000.0, e=1.0, pos=np.zeros((0, 2)), vel=np.zeros((0, 2)), rho_g=1.0,
        mu_g=nu, body_accel=(0.0, body_accel, 0.0), wall_u=wall_u, cs_smag=cs_smag,
        storage=storage)


def scaled_riser2d(nx=64, ny=128, n_particles=None, seed=SEED_BASE + 1,
                   storage=STORE_F32, **kw) -> Workload:
    """Riser section at the same solid fraction and cell size ratio as the
    256x2048 riser but a smaller lattice (for tests)."""
    if n_particles is None:
        n_particles = int(round(200000 * nx * ny / (256 * 2048)))
    return riser2d(nx=nx, ny=ny, n_particles=n_particles, seed=seed, storage=storage, **kw)


def scaled_riser3d(nx=32, ny=32, nz=64, n_particles=None, seed=SEED_BASE + 3,
                   storage=STORE_F32, **kw) -> Workload:
    if n_particles is None:
        n_particles = int(round(4000000 * nx * ny * nz / (256 * 256 * 1024)))
    return riser3d(nx=nx, ny=ny, nz=nz, n_particles=n_particles, seed=seed,
                   storage=storage, **kw)
