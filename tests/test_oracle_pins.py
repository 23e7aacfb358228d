"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden, with citations), closed-form flows, exact
conservation laws, textbook limits and brute force on small inputs.  None of
these tests needs a GPU.
"""
import json
import math
import os
import types

import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_2653_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def _sig_close(value, printed, digits):
    """value rounds to `printed` at the number of significant digits printed."""
    if printed == 0:
        return abs(value) < 10 ** -digits
    e = math.floor(math.log10(abs(printed)))
    return abs(value - printed) <= 0.5 * 10 ** (e - digits + 1) * (1 + 1e-9)


def _bed(**kw):
    base = dict(dim=2, n=(8, 8), bc=(W.WALL, W.WALL, W.PERIODIC, W.PERIODIC, W.PERIODIC,
                                     W.PERIODIC),
                h=1.0, dt=1.0, d_p=0.2, rho_s=1000.0, e=0.9, pos=np.zeros((0, 2)),
                vel=np.zeros((0, 2)), rho_g=1.0, mu_g=0.1, g=(0.0, 0.0, 0.0),
                body_accel=(0.0, 0.0, 0.0), u0=(0.0, 0.0, 0.0), inlet_u=None, wall_u=None,
                cs_smag=0.0, superficial_mode=0, pressure_plus=0)
    base.update(kw)
    return types.SimpleNamespace(**base)


# ---------------------------------------------------------------- unit tables

def test_units_table1():
    g = _golden("table1_bubbling.json")
    si, pr, dig = g["si"], g["printed_dimensionless"], g["printed_significant_digits"]
    w = _bed(h=si["h"], dt=si["dt"], d_p=si["d_p"], rho_s=si["rho_s"], rho_g=si["rho_g"],
             mu_g=si["mu_g"], e=si["e"], u0=(0.0, si["v_mf"], 0.0))
    k = O.units(w)
    assert _sig_close(k["d"], pr["d_p"], dig["d_p"])
    assert _sig_close(k["u0_y"], pr["v_mf"], dig["v_mf"])
    assert _sig_close(k["rho_s"], pr["rho_s"], dig["rho_s"])
    assert _sig_close(k["mu"], pr["mu_g"], dig["mu_g"])
    assert k["e"] == pr["e"]
    # the injection velocity entry is garbled by a factor 10
    wi = _bed(h=si["h"], dt=si["dt"], u0=(0.0, si["v_inj"], 0.0))
    assert _sig_close(O.units(wi)["u0_y"], pr["v_inj_garbled"] / 10, 1)
    # Eq. 3: tau = 3 nu + 1/2 with dt = 1
    assert k["tau"] == pytest.approx(3 * pr["mu_g"] + 0.5, rel=1e-5)


def test_units_table2_and_area_fraction():
    g = _golden("table2_riser.json")
    si, pr, dig, lat = g["si"], g["printed_dimensionless"], g["printed_significant_digits"], g["lattice"]
    w = _bed(h=si["h"], dt=si["dt"], d_p=si["d_p"], rho_s=si["rho_s"], rho_g=si["rho_g"],
             mu_g=si["mu_g"], u0=(0.0, si["v_inlet"], 0.0))
    k = O.units(w)
    assert _sig_close(k["d"], pr["d_p"], dig["d_p"])
    assert _sig_close(k["u0_y"], pr["v_inlet"], dig["v_inlet"])
    assert _sig_close(k["rho_s"], pr["rho_s"], dig["rho_s"])
    assert _sig_close(k["mu"], pr["mu_g_garbled"] * 10, 2)
    # Eq. 10 deposition on the Table 2 lattice: the bed-mean solid fraction is
    # the printed initial solids volume fraction (2D area fraction).
    h, d_p = si["h"], si["d_p"]
    nx, ny, N = lat["W"], lat["H"], lat["N"]
    pos = W.rsa(2, (nx * h, ny * h), (0.5 * d_p, 0.0), (nx * h - 0.5 * d_p, ny * h), (0, 1),
                d_p * (1 + 1e-9), N, 1303099)
    bed = O.OracleBed(_bed(n=(nx, ny), h=h, dt=si["dt"], d_p=d_p, rho_s=si["rho_s"],
                           rho_g=si["rho_g"], mu_g=si["mu_g"], pos=pos,
                           vel=np.zeros_like(pos)))
    bed.step(1)
    eps_s = bed.field(O.F_EPS_S)
    ntot = bed.field(O.F_NTOT)
    assert ntot.sum() == N
    cap = math.pi / (2 * math.sqrt(3))
    assert eps_s.max() < cap            # no cell reaches the packing cap
    assert eps_s.mean() == pytest.approx(pr["theta_s"], rel=1e-3)


# ---------------------------------------------------------- closed-form pieces

def test_omega_printed_range():
    g = _golden("emms_omega_range.json")
    assert _sig_close(O.omega(g["max"]["eps_g"]), g["max"]["omega"], g["max"]["significant_digits"])
    assert _sig_close(O.omega(g["min"]["eps_g"]), g["min"]["omega"], g["min"]["significant_digits"])
    eps = np.linspace(0.7401, 0.97, 20001)
    om = np.array([O.omega(e) for e in eps])
    assert om.max() == pytest.approx(g["max"]["omega"], abs=5e-5)
    assert om.min() == pytest.approx(g["min"]["omega"], abs=5e-5)
    # the last branch reaches the uncorrected drag (omega = 1) at eps_g = 1
    assert O.omega(1.0) == pytest.approx(1.0, abs=1e-12)
    # reading R5: no correction in the Ergun regime
    assert O.omega(0.5) == 1.0 and O.omega(0.74) == 1.0


def test_gamma_limits():
    # Eq. 9: gamma = 0 for pure fluid and 1 for pure solid
    for tau in (0.5008, 0.51, 0.8, 1.7):
        assert O.gamma(0.0, tau) == 0.0
        assert O.gamma(1.0, tau) == pytest.approx(1.0, abs=1e-15)
        g = [O.gamma(e, tau) for e in np.linspace(0, 1, 101)]
        assert np.all(np.diff(g) > 0)
    # Eq. 9 in tau: a partially filled cell loses its solid weighting as tau
    # falls to 1/2 and approaches the solid fraction itself as tau grows
    for es in (0.1, 0.45, 0.9):
        assert O.gamma(es, 0.5) == 0.0
        assert O.gamma(es, 0.5 + 1e-12) == pytest.approx(0.0, abs=1e-10)
        assert O.gamma(es, 1e9) == pytest.approx(es, rel=1e-8)


def test_eps3d_packings():
    # Eq. 11 maps the empty cell to eps = 1 and 2D hexagonal close packing of
    # discs (area fraction pi/(2 sqrt 3)) to simple-cubic packing of spheres
    # (volume fraction pi/6).
    assert O.eps3d(1.0) == 1.0
    hexagonal = math.pi / (2 * math.sqrt(3))
    assert O.eps3d(1.0 - hexagonal) == pytest.approx(1.0 - math.pi / 6, abs=1e-14)


def _schiller_naumann_force(re, rho, slip, d):
    cd = 24.0 / re * (1 + 0.15 * re ** 0.687) if re < 1000 else 0.44
    return cd * math.pi * d * d / 8.0 * rho * slip * slip


@pytest.mark.parametrize("slip", [1e-9, 1e-3, 0.3, 30.0])
def test_beta_isolated_sphere(slip):
    # beta V_p/(1-eps) |u-v| -> the drag of one sphere as eps_g -> 1
    rho, mu, d = 1.2, 1.8e-5, 1e-4
    eps = 1.0 - 1e-9
    f = O.beta(eps, slip, rho, mu, d) * (math.pi * d ** 3 / 6) / (1 - eps) * slip
    re = rho * slip * d / mu
    assert f == pytest.approx(_schiller_naumann_force(re, rho, slip, d), rel=1e-6)
    if re < 1e-3:   # Stokes' law
        assert f == pytest.approx(3 * math.pi * mu * d * slip, rel=1e-3)


@pytest.mark.parametrize("eps", [0.7401, 0.76, 0.81, 0.9, 0.96])
@pytest.mark.parametrize("slip", [1e-3, 0.3, 30.0])
def test_beta_dilute_branch_carries_omega(eps, slip):
    # Eq. 19 above eps_g = 0.74: 3/4 (1-eps) eps rho C_d0 |u-v| / d times the
    # EMMS correction omega(eps) of Eq. 20, with C_d0 the Schiller-Naumann
    # coefficient at Re_p = eps rho |u-v| d / mu (Eq. 21-22)
    rho, mu, d = 1.2, 1.8e-5, 1e-4
    re = eps * rho * slip * d / mu
    cd = 24.0 / re * (1 + 0.15 * re ** 0.687) if re < 1000 else 0.44
    want = 0.75 * (1 - eps) * eps * rho * cd * slip / d * O.omega(eps)
    assert O.beta(eps, slip, rho, mu, d) == pytest.approx(want, rel=1e-12)
    assert O.omega(eps) != 1.0


@pytest.mark.parametrize("eps", [0.4, 0.55, 0.74])
def test_beta_ergun_pressure_drop(eps):
    # Ergun: dp/L = 150 mu (1-e)^2 U/(e^3 d^2) + 1.75 rho (1-e) U^2/(e^3 d) for
    # superficial velocity U; the gas-side force per volume is beta (U/eps).
    rho, mu, d, U = 1.2, 1.8e-5, 5e-4, 0.05
    slip = U / eps
    dpdl = O.beta(eps, slip, rho, mu, d) * slip / eps
    ergun = 150 * mu * (1 - eps) ** 2 * U / (eps ** 3 * d ** 2) + 1.75 * rho * (1 - eps) * U ** 2 / (eps ** 3 * d)
    assert dpdl == pytest.approx(ergun, rel=1e-12)


def test_binary_collision_laws():
    rng = np.random.default_rng(7)
    for dim in (2, 3):
        for _ in range(200):
            m1, m2 = rng.uniform(0.5, 3.0, 2)
            e = rng.uniform(0.0, 1.0)
            p1, p2 = rng.normal(size=dim), rng.normal(size=dim)
            v1, v2 = rng.normal(size=dim), rng.normal(size=dim)
            a1, a2 = O.binary_collision(dim, m1, m2, e, p1, p2, v1, v2)
            n = (p1 - p2) / np.linalg.norm(p1 - p2)
            # momentum conservation
            np.testing.assert_allclose(m1 * a1 + m2 * a2, m1 * v1 + m2 * v2, rtol=0, atol=1e-12)
            # restitution law on the normal relative velocity
            assert np.dot(a1 - a2, n) == pytest.approx(-e * np.dot(v1 - v2, n), abs=1e-12)
            # tangential relative velocity unchanged
            t_before = (v1 - v2) - np.dot(v1 - v2, n) * n
            t_after = (a1 - a2) - np.dot(a1 - a2, n) * n
            np.testing.assert_allclose(t_after, t_before, atol=1e-12)
            # kinetic energy loss 1/2 mu (1 - e^2) g_n^2
            ke0 = 0.5 * m1 * v1 @ v1 + 0.5 * m2 * v2 @ v2
            ke1 = 0.5 * m1 * a1 @ a1 + 0.5 * m2 * a2 @ a2
            mu_r = m1 * m2 / (m1 + m2)
            assert ke0 - ke1 == pytest.approx(0.5 * mu_r * (1 - e * e) * np.dot(v1 - v2, n) ** 2,
                                              abs=1e-12)
    # a wall is an infinitely heavy particle at rest: v_n -> -e v_n
    a1, a2 = O.binary_collision(2, 1.0, 1e30, 0.9, [0.1, 0.5], [0.0, 0.5], [-0.2, 0.3], [0.0, 0.0])
    assert a1[0] == pytest.approx(0.18, abs=1e-15) and a1[1] == 0.3


# ------------------------------------------------------------- closed-form flows

def _channel(dim, nx, nu, accel=0.0, top_u=0.0, periodic_n=4):
    if dim == 2:
        n = (nx, periodic_n)
        bc = (W.WALL, W.WALL, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC)
        body = (0.0, accel, 0.0)
        pos = np.zeros((0, 2))
    else:
        n = (nx, periodic_n, periodic_n)
        bc = (W.WALL, W.WALL, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC)
        body = (0.0, 0.0, accel)
        pos = np.zeros((0, 3))
    wall_u = np.zeros((6, 3))
    wall_u[1, dim - 1] = top_u
    return _bed(dim=dim, n=n, bc=bc, mu_g=nu, body_accel=body, wall_u=wall_u, pos=pos,
                vel=pos.copy())


@pytest.mark.parametrize("dim", [2, 3])
def test_poiseuille_exact_at_magic_tau(dim):
    # BGK + half-way bounce-back reproduces the parabola with walls exactly on
    # the cell faces when (tau - 1/2)^2 = 3/16 (the TRT "magic" parameter).
    tau = 0.5 + math.sqrt(3.0) / 4.0
    nu = (tau - 0.5) / 3.0
    nx, F = 12, 1e-6
    bed = O.OracleBed(_channel(dim, nx, nu, accel=F))
    bed.step(12000)
    u = bed.field(O.F_U)[:, dim - 1].reshape(-1, nx)   # rows of the periodic axes
    x = np.arange(nx) + 0.5
    exact = F / (2 * nu) * x * (nx - x)
    np.testing.assert_allclose(u, np.broadcast_to(exact, u.shape), rtol=1e-9, atol=0)


@pytest.mark.parametrize("dim,tau", [(2, 0.51), (2, 1.3), (3, 0.8)])
def test_poiseuille_second_difference(dim, tau):
    # away from the magic tau the interior still solves u'' = -F/(rho nu)
    nu = (tau - 0.5) / 3.0
    nx, F = 10, 1e-6
    bed = O.OracleBed(_channel(dim, nx, nu, accel=F))
    steps = int(min(60000, 40 * nx * nx / nu))
    bed.step(steps)
    u = bed.field(O.F_U)[:, dim - 1].reshape(-1, nx)[0]
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    np.testing.assert_allclose(d2, -F / nu, rtol=1e-8)
    rho = bed.field(O.F_RHO)
    np.testing.assert_allclose(rho, 1.0, atol=1e-12)


@pytest.mark.parametrize("dim,tau", [(2, 0.6), (2, 1.2), (3, 0.9)])
def test_couette_linear(dim, tau):
    nu = (tau - 0.5) / 3.0
    nx, U = 10, 1e-3
    bed = O.OracleBed(_channel(dim, nx, nu, top_u=U))
    bed.step(int(min(60000, 40 * nx * nx / nu)))
    u = bed.field(O.F_U)[:, dim - 1].reshape(-1, nx)
    x = np.arange(nx) + 0.5
    np.testing.assert_allclose(u, np.broadcast_to(U * x / nx, u.shape), rtol=1e-9, atol=1e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_inflow_outflow_fixed_point(dim):
    # with periodic sides, a uniform stream at the inlet velocity is an exact
    # steady state of the inlet/outlet conditions; the oracle must relax to it
    u_in = 2e-3
    if dim == 2:
        n = (6, 16)
        bc = (W.PERIODIC, W.PERIODIC, W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC)
        inlet = np.zeros((6, 2)); inlet[:, 1] = u_in
    else:
        n = (4, 4, 16)
        bc = (W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.INLET, W.OUTLET)
        inlet = np.zeros((16, 3)); inlet[:, 2] = u_in
    pos = np.zeros((0, dim))
    bed = O.OracleBed(_bed(dim=dim, n=n, bc=bc, mu_g=0.2, inlet_u=inlet, pos=pos, vel=pos))
    bed.step(6000)
    u = bed.field(O.F_U)
    np.testing.assert_allclose(u[:, dim - 1], u_in, rtol=1e-8)
    np.testing.assert_allclose(u[:, : dim - 1], 0.0, atol=1e-13)
    np.testing.assert_allclose(bed.field(O.F_RHO), 1.0, atol=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_inlet_populations_follow_the_profile(dim):
    # A velocity inlet fills each population that enters a bottom cell from
    # below with the equilibrium at density 1 and that cell's inlet velocity
    # (reading R9); directions whose source crosses a side wall bounce back.
    if dim == 2:
        n, bc = (7, 6), (W.WALL, W.WALL, W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC)
        c, w = _c2()
    else:
        n, bc = (5, 4, 6), (W.WALL, W.WALL, W.WALL, W.WALL, W.INLET, W.OUTLET)
        c, w = _c3()
    nface = int(np.prod(n[:-1]))
    rng = np.random.default_rng(11)
    inlet = rng.uniform(-2e-3, 2e-3, (nface, dim))
    inlet[:, -1] = rng.uniform(1e-3, 4e-3, nface)
    pos = np.zeros((0, dim))
    # h = 2, dt = 1/2: lattice velocities are the SI ones times dt / h = 1/4
    bed = O.OracleBed(_bed(dim=dim, n=n, bc=bc, h=2.0, dt=0.5, mu_g=0.2, inlet_u=4 * inlet,
                           pos=pos, vel=pos))

    def check(profile):
        f = bed.populations()
        checked = 0
        for j in range(nface):
            q = np.array([j % n[0], j // n[0]])[: dim - 1]
            for i in range(len(w)):
                src = q - c[i][: dim - 1]
                if c[i][-1] != 1 or np.any(src < 0) or np.any(src >= np.array(n[: dim - 1])):
                    continue
                cu = c[i] @ profile[j]
                want = w[i] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * profile[j] @ profile[j])
                assert f[i, j] == pytest.approx(want, rel=1e-14), (j, i)
                checked += 1
        assert checked > 2 * nface

    bed.step(1)
    check(inlet)
    # a new profile (the end of a jet pulse, §3.1), given in SI, applies from
    # the next step
    inlet2 = inlet[::-1].copy() * 0.5
    bed.set_inlet(4 * inlet2)
    bed.step(1)
    check(inlet2)


# -------------------------------------------------------- coupled-step invariants

def _small_riser(dim=2, cs=0.0, **kw):
    if dim == 2:
        w = W.scaled_riser2d(nx=24, ny=48, storage=W.STORE_F64, cs_smag=cs, **kw)
    else:
        w = W.scaled_riser3d(nx=10, ny=10, nz=20, storage=W.STORE_F64, cs_smag=cs, **kw)
    return w


def _dense_bed(dim=2, seed=5, n_particles=400, **kw):
    """A small walled, periodic bed with a solid fraction high enough that
    many cells hold several particles, and fast random particle motion."""
    if dim == 2:
        w = W.riser2d(nx=16, ny=32, n_particles=n_particles, seed=seed, storage=W.STORE_F64,
                      solid_fraction=0.25, sigma_v=0.6, **kw)
    else:
        w = W.riser3d(nx=6, ny=6, nz=12, n_particles=n_particles, seed=seed,
                      storage=W.STORE_F64, solid_fraction=0.2, sigma_v=0.6, **kw)
    return w


@pytest.mark.parametrize("dim,cs", [(2, 0.0), (2, 0.15), (3, 0.0), (3, 0.15)])
def test_mass_conserved_with_particles(dim, cs):
    # Eq. 23: sum_i Omega^s_i = 0 and sum_i (f_i - feq_i) = 0, bounce-back and
    # periodic faces conserve populations: the gas mass is invariant.
    w = _small_riser(dim, cs)
    bed = O.OracleBed(w)
    m0 = bed.stats()["mass"]
    bed.step(20)
    m1 = bed.stats()["mass"]
    assert abs(m1 - m0) <= 1e-14 * m0


def _pre_collision_state(bed):
    f = bed.populations()
    return f


@pytest.mark.parametrize("dim", [2, 3])
def test_velocity_solves_eq24_and_force_is_eq25(dim):
    # The oracle solves Eq. 24 in closed form; check the implicit equation
    # itself, with Omega^s from Eq. 7 evaluated at the oracle's u, and that
    # Eq. 25 equals rho u + rho v_s - 2 m.
    w = _dense_bed(dim)
    bed = O.OracleBed(w)
    bed.step(3)
    f = bed.populations()          # pre-collision populations of the next step
    bed.step(1)
    k = bed.constants()
    rho = bed.field(O.F_RHO)
    u = bed.field(O.F_U)
    vs = bed.field(O.F_VS)
    eps_s = bed.field(O.F_EPS_S)
    om = bed.field(O.F_OMEGA)
    fpg = bed.field(O.F_FPG)
    og = om * np.array([O.gamma(e, k["tau"]) for e in eps_s])
    if dim == 2:
        c = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
        wts = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    else:
        c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1],
                      [0, 0, -1], [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1],
                      [-1, 0, -1], [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1],
                      [0, -1, 1]])
        wts = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    opp = np.array([int(np.where((c == -ci).all(axis=1))[0][0]) for ci in c])

    def feq(r, vel):
        cu = vel @ c.T
        uu = (vel * vel).sum(axis=1, keepdims=True)
        return wts * r[:, None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)

    fc = f.T                                        # (cell, q)
    omega_s = fc[:, opp] - fc + feq(rho, vs) - feq(rho, u)[:, opp]
    fb = np.array([k["fb_x"], k["fb_y"], k["fb_z"]])[:dim]
    lhs = rho[:, None] * u
    rhs = (fc + 0.5 * og[:, None] * omega_s) @ c + 0.5 * fb
    scale = np.abs(lhs).max()
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13 * scale)
    m = fc @ c
    closed = og[:, None] * (rho[:, None] * u + rho[:, None] * vs - 2 * m)
    np.testing.assert_allclose(fpg, closed, rtol=0, atol=1e-14 * max(np.abs(fpg).max(), 1e-30))
    assert np.abs(fpg).max() > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_third_law_rescale(dim):
    # Eq. 27-29: summing the rescaled drag over the particles deposited in a
    # cell gives |F_p->g| per component (its sign is the pre-estimate's)
    bed = O.OracleBed(_dense_bed(dim))
    bed.step(2)
    ids, cs = bed.sorted_ids()              # cell list used by the next step
    bed.step(1)
    fd = bed.particle_diag(O.P_FD)          # id order
    fpre = bed.particle_diag(O.P_FPRE)
    fpg = bed.field(O.F_FPG)
    S = bed.field(O.F_SUM_PRE)
    A = bed.field(O.F_SUM_ABS_PRE)
    ncell = cs.size - 1
    counts = np.diff(cs)
    owner = np.repeat(np.arange(ncell), counts)     # cell of each sorted slot
    cell_of_id = np.empty(ids.size, dtype=np.int64)
    cell_of_id[ids] = owner
    checked = 0
    for a in range(dim):
        tot = np.bincount(cell_of_id, weights=fd[:, a], minlength=ncell)
        pre = np.bincount(cell_of_id, weights=fpre[:, a], minlength=ncell)
        np.testing.assert_allclose(pre, S[:, a], rtol=1e-12, atol=1e-300)
        ok = (counts > 0) & (np.abs(S[:, a]) > 1e-9 * A[:, a])
        np.testing.assert_allclose(np.abs(tot[ok]), np.abs(fpg[ok, a]), rtol=1e-9)
        np.testing.assert_array_equal(np.sign(tot[ok]), np.sign(S[ok, a]))
        checked += ok.sum()
    assert checked > 50


def test_ballistic_particle_without_slip():
    # gas at rest, a resting particle: no slip, so F_p->g = 0, the pre-estimate
    # is 0 and so is the rescaled drag (reading R12); Eq. 16 leaves effective
    # gravity only: v' = (1 - rho_g/rho_s) g dt, P' = P + v' dt.
    h, dt = 1e-3, 1e-3
    w = _bed(n=(8, 8), h=h, dt=dt, d_p=0.3e-3, rho_s=2000.0, rho_g=1.0, mu_g=1e-4,
             g=(0.0, -9.81, 0.0), pos=np.array([[4.3e-3, 5.7e-3]]), vel=np.zeros((1, 2)))
    bed = O.OracleBed(w)
    bed.step(1)
    P, v = bed.particles()
    gy = (1 - 1.0 / 2000.0) * -9.81 * dt * dt / h
    assert v[0, 0] == 0.0 and v[0, 1] == pytest.approx(gy, rel=1e-14)
    assert P[0, 0] == pytest.approx(4.3, rel=1e-15)
    assert P[0, 1] == pytest.approx(5.7 + gy, rel=1e-15)


# ---------------------------------------------------- binning and hard spheres

def _neighbour_bruteforce(P, v, n, periodic, d):
    """O(N^2) approaching contact pairs, minimum image on periodic axes."""
    N, dim = P.shape
    pairs = []
    for i in range(N):
        for j in range(i + 1, N):
            dx = P[i] - P[j]
            for a in range(dim):
                if periodic[a]:
                    L = n[a]
                    if dx[a] > 0.5 * L:
                        dx[a] -= L
                    elif dx[a] < -0.5 * L:
                        dx[a] += L
            d2 = 0.0
            for a in range(dim):
                d2 = d2 + dx[a] * dx[a]
            if not d2 < d * d:
                continue
            dot = 0.0
            for a in range(dim):
                dot = dot + dx[a] * (v[i, a] - v[j, a])
            if dot < 0:
                pairs.append((i, j))
    return np.array(sorted(pairs), dtype=np.int64).reshape(-1, 2)


def _packed_state(dim, n, N, d, seed):
    rng = np.random.default_rng(seed)
    box = np.array(n, dtype=float)
    # overlapping positions are allowed here: detection is a pure function
    P = rng.uniform(0, 1, size=(N, dim)) * box
    v = rng.normal(size=(N, dim)) * 0.1
    return P, v


@pytest.mark.parametrize("dim,n,N", [(2, (6, 7), 200), (3, (4, 5, 6), 200)])
def test_detection_matches_bruteforce(dim, n, N):
    if dim == 2:
        bc = (W.WALL, W.WALL, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC)
        periodic = (False, True)
    else:
        bc = (W.WALL, W.WALL, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC)
        periodic = (False, True, True)
    d = 0.9
    P, v = _packed_state(dim, n, N, d, 11 + dim)
    w = _bed(dim=dim, n=n, bc=bc, d_p=d, pos=np.zeros((0, dim)), vel=np.zeros((0, dim)))
    bed = O.OracleBed(w)
    bed.set_particles(P, v)
    bed.collide_particles()
    got = bed.pairs()
    want = _neighbour_bruteforce(P, v, n, periodic, d)
    assert want.shape[0] > 20
    np.testing.assert_array_equal(got, want)
    # partner choice: nearest approaching contact, ties to the smaller id
    best = bed.particle_diag(O.P_BEST).astype(np.int64)
    for i in range(N):
        cand = [j for (a, b) in want for j in ((b,) if a == i else (a,) if b == i else ())]
        if not cand:
            assert best[i] == -1
            continue
        def d2(j):
            dx = P[i] - P[j]
            for a in range(dim):
                if periodic[a]:
                    if dx[a] > 0.5 * n[a]:
                        dx[a] -= n[a]
                    elif dx[a] < -0.5 * n[a]:
                        dx[a] += n[a]
            s = 0.0
            for a in range(dim):
                s = s + dx[a] * dx[a]
            return s
        assert best[i] == min(cand, key=lambda j: (d2(j), j))


def test_partner_ties_go_to_the_smaller_id():
    # Reading R14: among approaching contacts at exactly the same distance the
    # one with the smaller id is chosen.  Coordinates and speeds are exact in
    # binary, so both squared distances are 1/64.  Group 1: particle 0 between
    # 2 (cell to its left, visited first) and 1 (its own cell); group 2:
    # particle 3 with 4 and 5, all three in one cell.
    u = 0.015625
    P = np.array([[4.0, 4.5], [4.125, 4.5], [3.875, 4.5],
                  [2.0, 2.0], [2.0, 2.125], [2.125, 2.0]])
    v = np.array([[0.0, 0.0], [-u, 0.0], [u, 0.0],
                  [0.0, 0.0], [0.0, -u], [-u, 0.0]])
    w = _bed(n=(8, 8), d_p=0.15, pos=np.zeros((0, 2)), vel=np.zeros((0, 2)))
    bed = O.OracleBed(w)
    bed.set_particles(P, v)
    bed.collide_particles()
    best = bed.particle_diag(O.P_BEST).astype(np.int64)
    np.testing.assert_array_equal(best, [1, 0, 0, 4, 3, 3])
    # the chosen pairs collide head on (Eq. 17-18, equal masses); the third
    # particle of each group chose a partner that chose another: untouched
    _, v1 = bed.particles()
    e = w.e
    np.testing.assert_array_equal(v1[[2, 5]], v[[2, 5]])
    np.testing.assert_allclose(v1[0], [-(1 + e) / 2 * u, 0.0], rtol=1e-14)
    np.testing.assert_allclose(v1[1], [-(1 - e) / 2 * u, 0.0], rtol=1e-14)
    np.testing.assert_allclose(v1[3], [0.0, -(1 + e) / 2 * u], rtol=1e-14)
    np.testing.assert_allclose(v1[4], [0.0, -(1 - e) / 2 * u], rtol=1e-14)


def test_resolution_momentum_and_walls():
    # mutual nearest pairs collide by Eq. 17-18, the rest bounce off walls:
    # total particle momentum changes only through wall contacts
    dim, n, N, d = 2, (6, 7), 150, 0.9
    P, v = _packed_state(dim, n, N, d, 3)
    w = _bed(dim=dim, n=n, d_p=d, e=0.8, pos=np.zeros((0, 2)), vel=np.zeros((0, 2)))
    bed = O.OracleBed(w)
    bed.set_particles(P, v)
    bed.collide_particles()
    P1, v1 = bed.particles()
    np.testing.assert_array_equal(P1, P)
    best = bed.particle_diag(O.P_BEST).astype(np.int64)
    wall = bed.particle_diag(O.P_WALL).astype(np.int64)
    mutual = np.array([best[i] >= 0 and best[best[i]] == i for i in range(N)])
    assert mutual.sum() >= 4
    untouched = ~mutual & (wall == 0)
    np.testing.assert_array_equal(v1[untouched], v[untouched])
    walled = ~mutual & (wall != 0)
    assert walled.sum() > 0
    for i in np.where(walled)[0]:
        for a in range(dim):
            if wall[i] & (3 << (2 * a)):
                assert v1[i, a] == pytest.approx(-0.8 * v[i, a], abs=1e-15)
            else:
                assert v1[i, a] == v[i, a]
    # pair momentum conserved (equal masses)
    for i in np.where(mutual)[0]:
        j = best[i]
        if i < j:
            np.testing.assert_allclose(v1[i] + v1[j], v[i] + v[j], atol=1e-15)


def test_sort_and_deposition_bruteforce():
    w = _dense_bed(2)
    bed = O.OracleBed(w)
    bed.step(2)
    P, v = bed.particles()
    nx, ny = w.n
    cell = np.floor(P[:, 0]).astype(np.int64) + nx * np.floor(P[:, 1]).astype(np.int64)
    order = np.lexsort((np.arange(len(cell)), cell))
    ids, cs = bed.sorted_ids()
    np.testing.assert_array_equal(ids, order)
    np.testing.assert_array_equal(cs, np.r_[0, np.cumsum(np.bincount(cell, minlength=nx * ny))])
    # the next step deposits from this cell list
    bed.step(1)   # deposition of step 3 used the state above
    ntot = bed.field(O.F_NTOT)
    vs = bed.field(O.F_VS)
    np.testing.assert_array_equal(ntot, np.bincount(cell, minlength=nx * ny))
    for a in range(2):
        sums = np.bincount(cell, weights=v[:, a], minlength=nx * ny)
        with np.errstate(invalid="ignore", divide="ignore"):
            mean = np.where(ntot > 0, sums / np.maximum(ntot, 1), 0.0)
        np.testing.assert_allclose(vs[:, a], mean, rtol=1e-14, atol=1e-18)
    r = bed.constants()["r"]
    np.testing.assert_allclose(bed.field(O.F_EPS_S),
                               np.minimum(ntot * math.pi * r * r, math.pi / (2 * math.sqrt(3))),
                               rtol=1e-15)


def test_mean_voidage_of_current_positions():
    # The bed-mean voidage reported after a step is that of the particle
    # positions at the end of the step (Eq. 10 counts, Eq. 11 mapping), not
    # of the deposition at its start.
    w = _dense_bed(2)
    bed = O.OracleBed(w)
    bed.step(3)
    P, _ = bed.particles()
    nx, ny = w.n
    cell = np.floor(P[:, 0]).astype(np.int64) + nx * np.floor(P[:, 1]).astype(np.int64)
    n = np.bincount(cell, minlength=nx * ny)
    r = bed.constants()["r"]
    es = np.minimum(n * math.pi * r * r, math.pi / (2 * math.sqrt(3)))
    expect = np.mean([O.eps3d(1.0 - e) for e in es])
    assert bed.stats()["mean_eps_g"] == pytest.approx(expect, rel=1e-14)
    # the deposition of the last step used the positions before the move
    assert np.any(bed.field(O.F_NTOT) != n)


def _c2():
    c = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return c, w


def _c3():
    """D3Q19 in storage order: rest, the six axis directions (+x, -x, +y, -y,
    +z, -z), then the twelve edge diagonals in opposite pairs (xy, xz, yz)."""
    c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
                  [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    return c, w


@pytest.mark.parametrize("dim", [2, 3])
def test_les_reduces_to_bgk_and_solves_quadratic(dim):
    if dim == 2:
        w0, w1 = _small_riser(2, 0.0), _small_riser(2, 0.2)
        c, wts = _c2()
    else:
        # three different sides, and Q_ab summed over all three axes
        mk = lambda cs: W.scaled_riser3d(nx=8, ny=6, nz=12, storage=W.STORE_F64, cs_smag=cs)
        w0, w1 = mk(0.0), mk(0.2)
        c, wts = _c3()
    b0, b1 = O.OracleBed(w0), O.OracleBed(w1)
    b0.step(1)
    np.testing.assert_array_equal(b0.field(O.F_TAU_T), b0.constants()["tau"])
    # tau_t from Eq. 13-14: tau_t^2 - tau tau_t - 9 Cs^2 Q / (2 rho) = 0
    b1.step(5)
    f = b1.populations()
    b1.step(1)
    tau = b1.constants()["tau"]
    tt = b1.field(O.F_TAU_T)
    rho = b1.field(O.F_RHO)
    u = b1.field(O.F_U)[:, :dim]
    cu = u @ c.T
    uu = (u * u).sum(axis=1, keepdims=True)
    fe = wts * rho[:, None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
    neq = f.T - fe
    Q = np.einsum("xi,ia,ib->xab", neq, c, c)
    Qn = np.sqrt(2 * (Q * Q).sum(axis=(1, 2)))
    resid = tt * tt - tau * tt - 9 * 0.2 ** 2 * Qn / (2 * rho)
    np.testing.assert_allclose(resid, 0.0, atol=1e-14)
    assert (tt > tau).all() and (tt - tau).max() > 1e-9


# ------------------------------------------------ interpolation and integration

def test_pressure_force_interpolates_quadratic_density():
    # Gas at rest with rho = 1 + a (x-x0)^2 + b (y-y0)^2 and resting particles:
    # no slip, so the drag vanishes and Eq. 16 leaves -V_p grad p / m.  Central
    # differences of p = rho/3 at cell-centre nodes give a grad p linear in
    # position, which bilinear interpolation reproduces exactly:
    # grad p = (2a (x-x0), 2b (y-y0)) / 3 at the particle centre.
    nx, ny, a, b, x0, y0 = 16, 12, 2e-4, -3e-4, 7.3, 5.1
    rng = np.random.default_rng(3)
    P = np.column_stack([rng.uniform(1.5, nx - 1.5, 40), rng.uniform(1.5, ny - 1.5, 40)])
    keep = [0]
    for i in range(1, len(P)):
        if np.min(np.linalg.norm(P[keep] - P[i], axis=1)) > 0.25:
            keep.append(i)
    P = P[keep]
    wl = _bed(n=(nx, ny), bc=(W.WALL,) * 4 + (W.PERIODIC,) * 2, d_p=0.2, rho_s=500.0,
              pos=P, vel=np.zeros_like(P))
    bed = O.OracleBed(wl)
    c, w = _c2()
    xs = (np.arange(nx * ny) % nx) + 0.5
    ys = (np.arange(nx * ny) // nx) + 0.5
    rho = 1 + a * (xs - x0) ** 2 + b * (ys - y0) ** 2
    bed.set_populations(w[:, None] * rho[None, :])
    bed.step(1)
    P1, v1 = bed.particles()
    want = -np.column_stack([2 * a * (P[:, 0] - x0), 2 * b * (P[:, 1] - y0)]) / 3.0 / 500.0
    np.testing.assert_allclose(v1, want, rtol=1e-9, atol=1e-20)
    np.testing.assert_allclose(P1, P + v1, rtol=0, atol=1e-15)
    # the printed sign of Eq. 16 flips the force
    bed2 = O.OracleBed(_bed(**{**vars(wl), "pressure_plus": 1}))
    bed2.set_populations(w[:, None] * rho[None, :])
    bed2.step(1)
    np.testing.assert_allclose(bed2.particles()[1], -want, rtol=1e-9, atol=1e-20)


def test_pressure_force_interpolates_quadratic_density_3d():
    # The same on D3Q19 with trilinear weights, in a box whose three sides
    # differ (a z stride or node index built from the wrong side reads other
    # nodes): grad p = 2 (a_x (x-x0), a_y (y-y0), a_z (z-z0)) / 3.
    n, a, x0 = (10, 7, 12), np.array([2e-4, -3e-4, 1.5e-4]), np.array([4.3, 3.1, 6.7])
    rng = np.random.default_rng(4)
    P = np.column_stack([rng.uniform(1.5, n[k] - 1.5, 60) for k in range(3)])
    keep = [0]
    for i in range(1, len(P)):
        if np.min(np.linalg.norm(P[keep] - P[i], axis=1)) > 0.25:
            keep.append(i)
    P = P[keep]
    bed = O.OracleBed(_bed(dim=3, n=n, bc=(W.WALL,) * 6, d_p=0.2, rho_s=500.0, pos=P,
                           vel=np.zeros_like(P)))
    idx = np.arange(n[0] * n[1] * n[2])
    X = np.column_stack([idx % n[0], (idx // n[0]) % n[1], idx // (n[0] * n[1])]) + 0.5
    rho = 1 + ((X - x0) ** 2 * a).sum(axis=1)
    _, w = _c3()
    bed.set_populations(w[:, None] * rho[None, :])
    bed.step(1)
    P1, v1 = bed.particles()
    want = -2 * a * (P - x0) / 3.0 / 500.0
    np.testing.assert_allclose(v1, want, rtol=1e-9, atol=1e-20)
    np.testing.assert_allclose(P1, P + v1, rtol=0, atol=1e-15)


def test_close_packing_cap_3d():
    # Eq. 10 in 3D: eps_s = n V_p / h^3 up to the close packing of spheres,
    # pi / (3 sqrt 2); two spheres of d = 0.9 h in one cell would fill 0.76 of
    # it.  In 3D the gas voidage is 1 - eps_s (no Eq. 11).
    n = (7, 5, 5)
    P = np.array([[2.05, 2.05, 2.05], [2.95, 2.95, 2.95], [4.5, 2.5, 2.5]])
    bed = O.OracleBed(_bed(dim=3, n=n, bc=(W.WALL,) * 6, d_p=0.9, rho_s=500.0, pos=P,
                           vel=np.zeros_like(P)))
    bed.step(1)
    es, eg = bed.field(O.F_EPS_S), bed.field(O.F_EPS_G)
    two, one = 2 + n[0] * (2 + n[1] * 2), 4 + n[0] * (2 + n[1] * 2)
    vp = math.pi * 0.9 ** 3 / 6
    assert 2 * vp > math.pi / (3 * math.sqrt(2))
    assert es[two] == pytest.approx(math.pi / (3 * math.sqrt(2)), rel=1e-15)
    assert es[one] == pytest.approx(vp, rel=1e-15)
    np.testing.assert_allclose(eg, 1.0 - es, rtol=0, atol=1e-15)
    assert np.count_nonzero(es) == 2


def test_pre_drag_at_node_and_face_midpoint():
    # A particle on a node (cell centre) sees that node's values; one on the
    # face between two nodes sees their average (bilinear weights 1/2, 1/2).
    w = _dense_bed(2)
    bed = O.OracleBed(w)
    bed.step(3)
    P, v = bed.particles()
    nx = w.n[0]
    k = bed.constants()
    P[0] = [5.5, 9.5]
    P[1] = [8.0, 14.5]
    for i in (0, 1):   # keep the two probes clear of everybody else
        far = np.linalg.norm(P - P[i], axis=1) > 1.2
        far[i] = True
        far[:2] = True
        P, v = P[far], v[far]
    bed.set_particles(P, v)
    bed.step(1)
    fpre = bed.particle_diag(O.P_FPRE)
    uact = bed.field(O.F_UACT)
    beta = bed.field(O.F_BETA)
    eps = bed.field(O.F_EPS_G)
    vs = bed.field(O.F_VS)
    # node wiring of Eq. 19: eps_g (Eq. 11) and the actual-velocity slip
    slip = np.linalg.norm(uact - vs, axis=1)
    bnode = np.array([O.beta(e, s, 1.0, k["mu"], k["d"]) for e, s in zip(eps, slip)])
    np.testing.assert_allclose(beta, bnode, rtol=1e-15, atol=0)
    x0 = 5 + nx * 9
    want0 = k["vp"] * beta[x0] / (1 - eps[x0]) * (uact[x0] - v[0])
    np.testing.assert_allclose(fpre[0], want0, rtol=1e-13)
    xa, xb = 7 + nx * 14, 8 + nx * 14
    bm, em, um = 0.5 * (beta[xa] + beta[xb]), 0.5 * (eps[xa] + eps[xb]), 0.5 * (uact[xa] + uact[xb])
    want1 = k["vp"] * bm / (1 - em) * (um - v[1])
    np.testing.assert_allclose(fpre[1], want1, rtol=1e-13)


def test_specular_wall_and_periodic_wrap():
    # gas and particles move together (no slip, no actual-velocity conversion)
    # so the drag vanishes; one particle crosses the x- wall within the step,
    # one crosses the periodic y seam.
    U = np.array([-0.05, 0.04])
    nx, ny = 8, 8
    P = np.array([[0.03, 3.5], [4.5, 7.98]])
    wl = _bed(n=(nx, ny), d_p=0.2, rho_s=800.0, e=0.7, superficial_mode=2,
              pos=P, vel=np.tile(U, (2, 1)))
    bed = O.OracleBed(wl)
    c, w = _c2()
    cu = c @ U
    f = w * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * U @ U)
    bed.set_populations(np.repeat(f[:, None], nx * ny, axis=1))
    bed.step(1)
    P1, v1 = bed.particles()
    x1 = 0.03 + U[0]
    assert P1[0, 0] == pytest.approx(-x1, abs=1e-15)
    assert v1[0, 0] == pytest.approx(-0.7 * U[0], abs=1e-15)
    assert v1[0, 1] == pytest.approx(U[1], abs=1e-15)
    assert P1[1, 1] == pytest.approx(7.98 + 0.04 - ny, abs=1e-13)
    np.testing.assert_allclose(v1[1], U, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sign", [1, -1])
def test_specular_walls_and_periodic_seams_on_every_face(dim, sign):
    # As above on both faces of every axis: x walls, a periodic y seam, and in
    # 3D z walls.  Particles move with the gas, so the drag vanishes; the one
    # that leaves through a wall is mirrored back with v_n -> -e v_n, the one
    # that leaves through the seam re-enters on the other side unchanged.
    e = 0.7
    if dim == 2:
        n = (8, 8)
        bc = (W.WALL, W.WALL, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC)
        U = sign * np.array([-0.05, 0.04])
        P = (np.array([[0.03, 3.5], [4.5, 7.98]]) if sign > 0 else
             np.array([[7.97, 3.5], [4.5, 0.02]]))
        c, w = _c2()
    else:
        n = (6, 6, 6)
        bc = (W.WALL, W.WALL, W.PERIODIC, W.PERIODIC, W.WALL, W.WALL)
        U = sign * np.array([-0.05, 0.04, 0.03])
        P = (np.array([[0.03, 3.5, 3.5], [3.5, 5.98, 2.5], [2.5, 1.5, 5.98]]) if sign > 0 else
             np.array([[5.97, 3.5, 3.5], [3.5, 0.02, 2.5], [2.5, 1.5, 0.02]]))
        c, w = _c3()
    wl = _bed(dim=dim, n=n, bc=bc, d_p=0.2, rho_s=800.0, e=e, superficial_mode=2, pos=P,
              vel=np.tile(U, (len(P), 1)))
    bed = O.OracleBed(wl)
    cu = c @ U
    f = w * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * U @ U)
    bed.set_populations(np.repeat(f[:, None], int(np.prod(n)), axis=1))
    bed.step(1)
    P1, v1 = bed.particles()
    want_P, want_v = P + U, np.tile(U, (len(P), 1))
    for a in range(dim):
        L = n[a]
        for k in range(len(P)):
            x = want_P[k, a]
            if bc[2 * a] == W.PERIODIC:
                want_P[k, a] = x - L if x >= L else (x + L if x < 0 else x)
            elif x < 0 or x >= L:
                want_P[k, a] = -x if x < 0 else 2 * L - x
                want_v[k, a] = -e * U[a]
    crossed = (P + U < 0) | (P + U >= np.array(n))
    assert crossed.sum() == dim
    np.testing.assert_allclose(P1, want_P, rtol=0, atol=1e-13)
    np.testing.assert_allclose(v1, want_v, rtol=0, atol=1e-15)


def test_pressure_gradient_at_walls_and_across_a_periodic_seam():
    # rho = 1 + a (x - x0)^2 + b cos(2 pi y / ny), gas at rest, walls in x,
    # periodic in y.  Node x-gradient of p = rho/3: 2a (x - x0)/3 inside, the
    # one-sided 2a (1 - x0)/3 and 2a (nx - 1 - x0)/3 on the wall nodes (exact
    # for a quadratic); node y-gradient, the wrap included:
    # -b sin(2 pi y / ny) sin(2 pi / ny) / 3.  A particle within half a cell
    # of a wall sees the wall node alone; one within half a cell of the seam
    # blends the last and the first node row.
    nx, ny, a, b, x0 = 12, 10, 2e-4, 3e-4, 5.3
    gy = lambda y: -b * np.sin(2 * np.pi * y / ny) * np.sin(2 * np.pi / ny) / 3
    P = np.array([[0.3, 4.5], [nx - 0.3, 6.5], [5.5, 0.2], [7.5, ny - 0.2]])
    bc = (W.WALL, W.WALL, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC)
    bed = O.OracleBed(_bed(n=(nx, ny), bc=bc, d_p=0.2, rho_s=500.0, pos=P,
                           vel=np.zeros_like(P)))
    xs = (np.arange(nx * ny) % nx) + 0.5
    ys = (np.arange(nx * ny) // nx) + 0.5
    rho = 1 + a * (xs - x0) ** 2 + b * np.cos(2 * np.pi * ys / ny)
    _, w = _c2()
    bed.set_populations(w[:, None] * rho[None, :])
    bed.step(1)
    g = bed.field(O.F_GRADP)
    gx = 2 * a * (xs - x0) / 3
    gx[xs == 0.5] = 2 * a * (1 - x0) / 3
    gx[xs == nx - 0.5] = 2 * a * (nx - 1 - x0) / 3
    np.testing.assert_allclose(g[:, 0], gx, rtol=1e-9, atol=1e-20)
    np.testing.assert_allclose(g[:, 1], gy(ys), rtol=1e-9, atol=1e-20)
    want = -np.array([
        [2 * a * (1 - x0) / 3, gy(4.5)],
        [2 * a * (nx - 1 - x0) / 3, gy(6.5)],
        [2 * a * (5.5 - x0) / 3, 0.3 * gy(-0.5) + 0.7 * gy(0.5)],
        [2 * a * (7.5 - x0) / 3, 0.7 * gy(ny - 0.5) + 0.3 * gy(0.5)]]) / 500.0
    np.testing.assert_allclose(bed.particles()[1], want, rtol=1e-9, atol=1e-20)


@pytest.mark.parametrize("dim", [2, 3])
def test_global_momentum_balance_periodic_box(dim):
    # In a fully periodic box streaming preserves total momentum, so the gas
    # momentum change over one step is the sum over cells of the collision's
    # momentum change: -(1-gamma(eps_s,tau_t))/tau_t (m - rho u) + F_p->g
    # + (1 - 1/(2 tau_t)) F_b  (Eq. 23 with Guo's source).  LES is on so that
    # tau_t differs from tau.
    w = _dense_bed(dim, cs_smag=0.3)
    w = w.with_(bc=(W.PERIODIC,) * 6)
    bed = O.OracleBed(w)
    bed.step(2)
    f = bed.populations()
    p0 = bed.stats()["gas_momentum"][:dim]
    bed.step(1)
    p1 = bed.stats()["gas_momentum"][:dim]
    k = bed.constants()
    rho = bed.field(O.F_RHO)
    u = bed.field(O.F_U)
    tt = bed.field(O.F_TAU_T)
    eps_s = bed.field(O.F_EPS_S)
    fpg = bed.field(O.F_FPG)
    assert (tt - k["tau"]).max() > 1e-6
    if dim == 2:
        c = _c2()[0]
    else:
        c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1],
                      [0, 0, -1], [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1],
                      [-1, 0, -1], [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1],
                      [0, -1, 1]])
    m = f.T @ c
    gt = np.array([O.gamma(e, t) for e, t in zip(eps_s, tt)])
    fb = np.array([k["fb_x"], k["fb_y"], k["fb_z"]])[:dim]
    dm = (-(1 - gt) / tt)[:, None] * (m - rho[:, None] * u) + fpg + (1 - 0.5 / tt)[:, None] * fb
    np.testing.assert_allclose(p1 - p0, dm.sum(axis=0), rtol=1e-9, atol=1e-15)
    # and the relaxation term really is present
    assert np.abs((-(1 - gt) / tt)[:, None] * (m - rho[:, None] * u)).sum() > 1e-3 * np.abs(dm).sum()


@pytest.mark.parametrize("dim", [2, 3])
def test_statistics_are_the_sums_of_the_state(dim):
    # The FP64 statistics of a step (spec reductions): gas mass and
    # momentum are sum_i f_i and sum_i c_i f_i over all cells, the particle
    # momentum is m_p sum_k v_k, and the mean slip is the particle-weighted
    # mean over occupied cells of |u_act - v_s| from the step's deposition.
    # Recomputed here with exactly rounded sums.
    w = _dense_bed(dim)
    bed = O.OracleBed(w)
    bed.step(3)
    st = bed.stats()
    f = bed.populations()
    c, _ = _c2() if dim == 2 else _c3()
    assert st["mass"] == pytest.approx(math.fsum(f.ravel()), rel=1e-15)
    for a in range(dim):
        ga = math.fsum((c[:, a][:, None] * f).ravel())
        assert st["gas_momentum"][a] == pytest.approx(ga, rel=1e-12, abs=1e-15)
    _, v = bed.particles()
    mp = bed.constants()["mp"]
    np.testing.assert_allclose(st["particle_momentum"][:dim],
                               [mp * math.fsum(v[:, a]) for a in range(dim)], rtol=1e-12)
    n = bed.field(O.F_NTOT).astype(float)
    slip = np.linalg.norm(bed.field(O.F_UACT)[:, :dim] - bed.field(O.F_VS)[:, :dim], axis=1)
    assert (n > 1).any() and (n == 0).any()
    assert st["mean_slip"] == pytest.approx(math.fsum(n * slip) / math.fsum(n), rel=1e-13)
    assert st["mean_slip"] > 0


def test_touching_spheres_without_approach_do_not_collide():
    # §2.2: a contact collides only when (P1-P2).(v1-v2) is negative; equal
    # velocities (zero product) or separating spheres do not collide.
    P = np.array([[2.5, 2.5], [2.9, 2.5], [4.5, 4.5], [4.9, 4.5]])
    v = np.array([[0.01, 0.02], [0.01, 0.02], [-0.01, 0.0], [0.01, 0.0]])
    bed = O.OracleBed(_bed(n=(8, 8), d_p=0.5, pos=np.zeros((0, 2)), vel=np.zeros((0, 2))))
    bed.set_particles(P, v)
    bed.collide_particles()
    assert bed.pairs().shape[0] == 0
    np.testing.assert_array_equal(bed.particles()[1], v)
    # reversing the second pair makes it approach
    v[2, 0], v[3, 0] = 0.01, -0.01
    bed.set_particles(P, v)
    bed.collide_particles()
    np.testing.assert_array_equal(bed.pairs(), [[2, 3]])


def _cfb_column(nx=16, ny=40, n=60, seed=9, vy=0.35, storage=W.STORE_F64):
    """Circulating-bed column (inlet below, outlet above, solids loop closed)
    with every particle moving up at vy lattice units per step."""
    w = W.cfb_riser2d(nx=nx, ny=ny, n_particles=n, seed=seed, storage=storage, cs_smag=0.0)
    vel = np.zeros_like(w.pos)
    vel[:, 1] = vy * w.h / w.dt
    return w.with_(vel=vel)


def test_recirculation_wraps_outlet_crossings_and_counts_them():
    # Reading R21: a particle whose move takes it through the outlet re-enters
    # through the inlet at the same lateral position and velocity; the count
    # of such crossings is the solids flux of §3.2 in particles.
    w = _cfb_column()
    bed = O.OracleBed(w)
    L = float(w.n[1])
    seen = 0
    for _ in range(30):
        P0, _ = bed.particles()
        out0 = bed.stats()["solids_out"]
        bed.step(1)
        P1, v1 = bed.particles()
        # no contact changed a velocity after the move (all move alike)
        assert len(bed.pairs()) == 0
        y = P0[:, 1] + v1[:, 1]
        crossed = y >= L
        np.testing.assert_array_equal(P1[:, 1], np.where(crossed, y - L, y))
        np.testing.assert_array_equal(P1[:, 0], P0[:, 0] + v1[:, 0])
        assert bed.stats()["solids_out"] - out0 == int(crossed.sum())
        seen += int(crossed.sum())
    # 60 particles at 0.35 cells per step over 40 cells: each crosses about
    # 30 * 0.35 / 40 times
    assert seen > 0
    assert bed.np == w.n_particles


def test_recirculation_needs_inlet_below_and_outlet_above():
    w = _cfb_column()
    with pytest.raises(Exception):
        O.OracleBed(w.with_(bc=(W.WALL, W.WALL, W.OUTLET, W.INLET, W.PERIODIC, W.PERIODIC)))


def _counted_bed(counts, storage=W.STORE_F64):
    """A Table 1 bed whose cell (x, y) holds counts[y, x] particles on a 4 x 4
    sub-grid of the cell (spacing 0.25 > d = 0.2, so no two overlap)."""
    ny, nx = counts.shape
    w = W.bubbling_table1(nx=nx, ny=ny, n_particles=1, storage=storage)
    pts = []
    for y in range(ny):
        for x in range(nx):
            for k in range(int(counts[y, x])):
                pts.append((x + 0.125 + 0.25 * (k % 4), y + 0.125 + 0.25 * (k // 4)))
    pos = np.array(pts, dtype=np.float64).reshape(-1, 2) * w.h
    return w.with_(pos=pos, vel=np.zeros_like(pos))


def _scipy_bubbles(mask):
    # independent reference: scipy's 4-connected labelling, regions touching
    # the top row left out
    ndimage = pytest.importorskip("scipy.ndimage")
    lab, n = ndimage.label(mask)
    top = set(lab[-1][lab[-1] > 0].tolist())
    sizes = [int((lab == k).sum()) for k in range(1, n + 1) if k not in top]
    return {"largest": max(sizes, default=0), "count": len(sizes), "cells": sum(sizes)}


def test_bubbles_of_a_designed_bed():
    # §3.1: regions with voidage above 0.85; two holes in a packed bed, the
    # empty freeboard above it is not a bubble
    counts = np.full((24, 12), 16)
    counts[-5:, :] = 0                 # freeboard
    counts[6:9, 4:7] = 0               # 3 x 3 hole
    counts[0, 9:11] = 0                # 2 x 1 hole on the bottom row
    bed = O.OracleBed(_counted_bed(counts))
    assert bed.bubbles(0.85) == {"largest": 9, "count": 2, "cells": 11}


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bubbles_match_scipy_labelling(seed):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 17, size=(30, 14))
    counts[rng.random(counts.shape) < 0.35] = 0
    w = _counted_bed(counts)
    bed = O.OracleBed(w)
    r = 0.5 * w.d_p / w.h
    eps2d = 1.0 - np.minimum(counts * math.pi * r * r, math.pi / (2 * math.sqrt(3)))
    assert bed.bubbles(0.85, 0) == _scipy_bubbles(eps2d > 0.85)
    # Eq. 11 voidage, written out independently
    epsg = 1.0 - math.sqrt(2.0) / math.sqrt(math.pi * math.sqrt(3.0)) * (1.0 - eps2d) ** 1.5
    assert bed.bubbles(0.97, 1) == _scipy_bubbles(epsg > 0.97)


def _counted_bed3d(counts, periodic_x=False, storage=W.STORE_F64):
    """A closed 3D box of Table 1 particles whose cell (x, y, z) holds
    counts[z, y, x] centres on a 3 x 3 x 3 sub-grid of the cell (spacing h/3
    > d_p, so no two overlap); x optionally periodic."""
    nz, ny, nx = counts.shape
    w = W.packed_bed(dim=3, n=(nx, ny, nz), n_particles=1, storage=storage)
    pts = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for k in range(int(counts[z, y, x])):
                    s = (k % 3, (k // 3) % 3, k // 9)
                    pts.append((x + (s[0] + 0.5) / 3, y + (s[1] + 0.5) / 3, z + (s[2] + 0.5) / 3))
    pos = np.array(pts, dtype=np.float64).reshape(-1, 3) * w.h
    bc = list(w.bc)
    if periodic_x:
        bc[0] = bc[1] = W.PERIODIC
    return w.with_(pos=pos, vel=np.zeros_like(pos), bc=tuple(bc))


def _scipy_bubbles_wrapped(mask, wrap_axes=()):
    """scipy's face-connected labelling of a (z, y, x) mask, then the labels
    that face each other across a periodic axis merged (union-find), then the
    regions reaching the top z layer left out."""
    ndimage = pytest.importorskip("scipy.ndimage")
    lab, n = ndimage.label(mask)
    parent = list(range(n + 1))

    def find(k):
        while parent[k] != k:
            parent[k] = parent[parent[k]]
            k = parent[k]
        return k

    for ax in wrap_axes:
        a = np.take(lab, 0, axis=ax)
        b = np.take(lab, -1, axis=ax)
        for p, q in zip(a[(a > 0) & (b > 0)].tolist(), b[(a > 0) & (b > 0)].tolist()):
            parent[find(p)] = find(q)
    root = np.array([find(k) for k in range(n + 1)])[lab]
    top = set(root[-1][lab[-1] > 0].tolist())
    sizes = [int((root == k).sum()) for k in set(root[lab > 0].tolist()) if k not in top]
    return {"largest": max(sizes, default=0), "count": len(sizes), "cells": sum(sizes)}


@pytest.mark.parametrize("seed,periodic_x", [(4, False), (5, False), (6, True), (7, True)])
def test_bubbles_match_scipy_labelling_3d(seed, periodic_x):
    # §3.1 regions in a 3D bed: face neighbours only, the vertical axis is z,
    # Eq. 10-11 in 3D is eps_g = 1 - n V_p / h^3 (below close packing)
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 28, size=(9, 6, 7))
    counts[rng.random(counts.shape) < 0.1] = 0
    w = _counted_bed3d(counts, periodic_x)
    bed = O.OracleBed(w)
    vp = math.pi * w.d_p ** 3 / 6.0 / w.h ** 3
    epsg = 1.0 - counts * vp
    # cells below 2.4, 3.6 and 6.0 centres: site fractions about 0.2 to 0.3,
    # under the percolation threshold of the cubic lattice, so many regions
    for thr in (0.99, 0.985, 0.975):
        got = bed.bubbles(thr, 1)
        assert got == _scipy_bubbles_wrapped(epsg > thr, (2,) if periodic_x else ())
        assert got["count"] >= 1
    # without the wrap the labelling of a periodic bed differs for some seed:
    # the merge across the x face is exercised, not vacuous
    if periodic_x:
        assert any(bed.bubbles(t, 1) != _scipy_bubbles_wrapped(epsg > t) for t in (0.99, 0.985, 0.975))


# ------------------------------------------------------- soft spheres (R25)

def _soft(dim=2, n=(16, 8), e=0.9, contact_steps=40.0, rho_s=1e6, **kw):
    """Lattice-unit bed (h = dt = rho_g = 1) with the soft-sphere model; the
    solid density is high so that the gas drag on the particles is negligible
    beside the contact forces (drag acceleration ~ 18 mu slip / (rho_s d^2))."""
    d = kw.pop("d_p", 0.5)
    mp = rho_s * math.pi * d ** 3 / 6.0
    kn = 0.5 * mp * (math.pi / contact_steps) ** 2
    base = dict(dim=dim, n=n, bc=(W.PERIODIC,) * 6, d_p=d, rho_s=rho_s, e=e, mu_g=0.1,
                collision_model=1, dem_kn=kn)
    base.update(kw)
    return _bed(**base), mp, kn


def _clipped_restitution(e):
    """Restitution and peak overlap of a continuous-time linear spring-dashpot
    contact whose force never pulls (F = max(0, k s + eta s')), integrated by
    scipy at tight tolerance: units m_eff = k = 1, approach speed 1."""
    integrate = pytest.importorskip("scipy.integrate")
    le = math.log(e)
    c = 2.0 * (-le / math.sqrt(math.pi ** 2 + le * le))

    def rhs(t, y):
        return [y[1], -max(0.0, y[0] + c * y[1])]

    def out(t, y):
        return y[0]
    out.terminal, out.direction = True, -1
    sol = integrate.solve_ivp(rhs, [0.0, 20.0], [0.0, 1.0], events=out, rtol=1e-12, atol=1e-14,
                              max_step=1e-3, dense_output=True)
    t_end = sol.t_events[0][0]
    ts = np.linspace(0.0, t_end, 4001)
    return -sol.y_events[0][0][1], sol.sol(ts)[0].max()


@pytest.mark.parametrize("e", [0.9, 0.5, 1.0])
def test_soft_sphere_pair_restitution(e):
    # A head-on pair with the damping that gives restitution e to a linear
    # spring-dashpot contact of reduced mass m/2: the separation speed and the
    # peak overlap match the continuous-time contact (no pulling force) up to
    # the time discretisation, and the error shrinks as the contact is
    # resolved by more steps.
    e_ref, s_ref = _clipped_restitution(e)
    errs = []
    for steps in (40.0, 160.0):
        w, mp, kn = _soft(e=e, contact_steps=steps)
        v = 1e-3
        P = np.array([[8 - 0.25 - 0.02, 4.3], [8 + 0.25 + 0.02, 4.3]])
        V = np.array([[v, 0.0], [-v, 0.0]])
        bed = O.OracleBed(w.__class__(**{**vars(w), "pos": P, "vel": V}))
        gap_min = np.inf
        for _ in range(int(3 * steps) + 60):
            bed.step(1)
            Pn, Vn = bed.particles()
            gap_min = min(gap_min, Pn[1, 0] - Pn[0, 0])
        e_num = (Vn[1, 0] - Vn[0, 0]) / (2 * v)
        overlap_ref = 2 * v * math.sqrt(0.5 * mp / kn) * s_ref
        assert abs((0.5 - gap_min) - overlap_ref) <= 0.05 * overlap_ref
        errs.append(abs(e_num - e_ref))
        # no lateral motion beyond what the disturbed gas gives; total
        # momentum kept up to the (negligible) drag
        assert np.abs(Vn[:, 1]).max() < 1e-6 * v
        assert abs(Vn[0, 0] + Vn[1, 0]) < 1e-3 * v
    assert errs[0] <= 0.015
    assert errs[1] <= 0.3 * errs[0] + 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_soft_sphere_rests_on_the_floor(dim):
    # A particle settles on the bottom wall where the spring carries its
    # effective weight: overlap = m_p g_eff / k_n.
    n = (8, 8) if dim == 2 else (6, 6, 8)
    g = 1e-5
    grav = (0.0, -g, 0.0) if dim == 2 else (0.0, 0.0, -g)
    P = np.full((1, dim), 3.4)
    P[0, -1] = 0.5
    w, mp, kn = _soft(dim=dim, n=n, e=0.3, contact_steps=40.0, bc=(W.WALL,) * 6, g=grav,
                      pos=P, vel=np.zeros((1, dim)))
    bed = O.OracleBed(w)
    bed.step(3000)
    Pn, Vn = bed.particles()
    g_eff = (1.0 - 1.0 / w.rho_s) * g
    assert Pn[0, -1] == pytest.approx(0.25 - mp * g_eff / kn, rel=1e-9)
    assert np.abs(Vn).max() < 1e-5 * g
    assert bed.particle_diag(O.P_FC)[0, -1] == pytest.approx(mp * g_eff, rel=1e-9)


def _soft_forces_bruteforce(P, v, n, per, d, kn, eta, eta_w, top_open=False):
    """All pairs (minimum image on periodic axes) and every face."""
    N, dim = P.shape
    r = 0.5 * d
    F = np.zeros((N, dim))
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            dx = P[i] - P[j]
            for a in range(dim):
                if per[a]:
                    dx[a] -= n[a] * round(dx[a] / n[a])
            dist = math.sqrt(dx @ dx)
            if dist >= d:
                continue
            nrm = dx / dist
            f = kn * (d - dist) - eta * ((v[i] - v[j]) @ nrm)
            F[i] += max(f, 0.0) * nrm
        for a in range(dim):
            if per[a]:
                continue
            if P[i, a] < r:
                F[i, a] += max(kn * (r - P[i, a]) - eta_w * v[i, a], 0.0)
            if not (top_open and a == dim - 1) and n[a] - P[i, a] < r:
                F[i, a] -= max(kn * (r - (n[a] - P[i, a])) + eta_w * v[i, a], 0.0)
    return F


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("walls", [False, True])
def test_soft_sphere_forces_match_all_pairs(dim, walls):
    # The contact forces from the cell neighbourhood equal those of an
    # all-pairs search; in a periodic box they sum to zero (third law).
    n = (7, 6) if dim == 2 else (5, 4, 6)
    rng = np.random.default_rng(11 + dim)
    d = 0.7
    box = np.array(n, dtype=float)
    pos = W.rsa(dim, box, [0.36] * dim, box - 0.36, (0, 0, 0) if walls else (1, 1, 1), 0.8 * d,
                60 if dim == 2 else 120, 5 + dim)
    vel = rng.normal(scale=2e-3, size=pos.shape)
    bc = (W.WALL,) * 6 if walls else (W.PERIODIC,) * 6
    w, mp, kn = _soft(dim=dim, n=n, d_p=d, rho_s=50.0, e=0.6, contact_steps=12.0, bc=bc,
                      pos=pos, vel=vel)
    bed = O.OracleBed(w)
    P0, v0 = bed.particles()
    k = bed.constants()
    bed.step(1)
    fc = bed.particle_diag(O.P_FC)
    ref = _soft_forces_bruteforce(P0, v0, n, [not walls] * dim, d, k["kn"], k["eta"], k["eta_w"])
    assert (np.abs(ref).sum(axis=1) > 0).mean() > 0.4
    np.testing.assert_allclose(fc, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    if not walls:
        assert np.abs(fc.sum(axis=0)).max() <= 1e-12 * np.abs(fc).sum()
    # and the force enters Eq. 16 like the drag: the particle momentum
    # changes by the contact, drag, pressure and gravity forces of the step
    assert k["eta"] == pytest.approx(k["eta_w"] / math.sqrt(2.0), rel=1e-14)


def test_soft_sphere_outlet_of_circulating_bed_is_open():
    # With the solids loop closed (R21) the outlet lets particles through, so
    # it exerts no contact force; the inlet face below still does.
    w = _cfb_column()
    r = 0.5 * w.d_p / w.h
    P = np.array([[4.5, w.n[1] - 0.5 * r], [8.5, 0.5 * r]])
    v = np.array([[0.0, 0.08], [0.0, -0.01]])
    w = W.soft_spheres(w, contact_steps=20.0).with_(pos=P * w.h, vel=v * w.h / w.dt)
    bed = O.OracleBed(w)
    bed.step(1)
    fc = bed.particle_diag(O.P_FC)
    assert fc[0, 1] == 0.0 and fc[0, 0] == 0.0
    assert fc[1, 1] > 0.0
    assert bed.stats()["solids_out"] == 1


# ------------------------------------------------ soft-sphere friction (R26)

def _cross(a, b):
    return np.cross(np.asarray(a, dtype=float), np.asarray(b, dtype=float))


@pytest.mark.parametrize("dim", [2, 3])
def test_friction_turns_sliding_into_rolling(dim):
    # A sphere set sliding on a floor (no spin) is slowed and spun up by
    # friction until its contact point stops slipping; the angular momentum
    # about the contact point is conserved meanwhile, so it rolls on at
    # v0 / (1 + I / (m l^2)) with l the lever arm (5/7 v0 for l = r), and its
    # contact point is then at rest.
    g, v0 = 1e-5, 1e-3
    d, rho_s, steps = 0.5, 1e9, 40.0
    mp = rho_s * math.pi * d ** 3 / 6.0
    kn = 0.5 * mp * (math.pi / steps) ** 2
    g_eff = (1.0 - 1.0 / rho_s) * g
    l = 0.25 - mp * g_eff / kn           # resting on its spring
    n = (16, 8) if dim == 2 else (16, 6, 8)
    P = np.full((1, dim), 3.0)
    P[0, -1] = l
    V = np.zeros((1, dim))
    V[0, 0] = v0
    grav = (0.0, -g, 0.0) if dim == 2 else (0.0, 0.0, -g)
    w, _, _ = _soft(dim=dim, n=n, e=0.3, contact_steps=steps, bc=(W.WALL,) * 6, g=grav, pos=P,
                    vel=V, rho_s=rho_s, dem_mu=0.5, dem_gamma_t=0.08 * mp)
    bed = O.OracleBed(w)
    bed.step(1500)
    Pn, Vn = bed.particles()
    spin = bed.spin()
    inertia = 0.4 * mp * 0.25 ** 2
    assert bed.constants()["inertia"] == pytest.approx(inertia, rel=1e-14)
    assert Pn[0, -1] == pytest.approx(l, rel=1e-9)
    assert Vn[0, 0] == pytest.approx(v0 / (1.0 + inertia / (mp * l * l)), rel=1e-6)
    # rolling: the contact point (at -l n below the centre) is at rest
    om = np.array([0.0, 0.0, spin[0]]) if dim == 2 else spin[0]
    nrm = np.zeros(3)
    nrm[dim - 1] = 1.0
    vel = np.zeros(3)
    vel[:dim] = Vn[0]
    vc = vel + _cross(om, -l * nrm)
    assert np.abs(vc).max() <= 1e-6 * v0
    # the slide lasted about (2/7) v0 / (mu g): far shorter than the run
    assert Vn[0, 0] < 0.75 * v0


@pytest.mark.parametrize("dim", [2, 3])
def test_friction_keeps_angular_momentum_of_a_pair(dim):
    # An oblique collision of two spinning spheres with friction: the contact
    # forces are equal and opposite and act at one point half way between the
    # centres, so the total angular momentum sum m P x v + I w about any point
    # is kept while the spins change.  The gas acts on the particles at a
    # relative rate of about 18 nu / (rho_s d^2) = 7e-9 per step: 1e-6 over
    # the run; a torque of the wrong sign or arm would change L by ~1e-1.
    d, rho_s = 0.5, 1e9
    n = (16, 12) if dim == 2 else (12, 12, 12)
    if dim == 2:
        P = np.array([[5.0, 6.0], [5.6, 6.2]])
        V = np.array([[1e-3, 0.0], [-1e-3, 0.0]])
    else:
        P = np.array([[5.0, 6.0, 6.0], [5.6, 6.2, 5.9]])
        V = np.array([[1e-3, 0.0, 2e-4], [-1e-3, 0.0, 0.0]])
    w, mp, kn = _soft(dim=dim, n=n, d_p=d, rho_s=rho_s, e=0.8, contact_steps=30.0, pos=P, vel=V,
                      dem_mu=0.4, dem_gamma_t=0.05 * rho_s * math.pi * d ** 3 / 6.0)
    bed = O.OracleBed(w)
    spin0 = np.array([2e-3, -1e-3]) if dim == 2 else np.array([[0.0, 1e-3, 2e-3], [-1e-3, 0.0, 0.0]])
    bed.set_spin(spin0)
    inertia = bed.constants()["inertia"]

    def ang(Pp, Vp, sp):
        P3 = np.zeros((2, 3)); V3 = np.zeros((2, 3))
        P3[:, :dim] = Pp; V3[:, :dim] = Vp
        om = np.column_stack([np.zeros(2), np.zeros(2), sp]) if dim == 2 else sp
        return (mp * np.cross(P3, V3)).sum(axis=0) + inertia * om.sum(axis=0)

    L0 = ang(*bed.particles(), bed.spin())
    bed.step(150)
    Pn, Vn = bed.particles()
    L1 = ang(Pn, Vn, bed.spin())
    assert np.abs(bed.spin() - spin0).max() > 1e-4          # friction acted
    assert np.abs(L1 - L0).max() <= 1e-6 * np.abs(L0).max()


def test_friction_off_reduces_to_the_normal_contact():
    # mu = 0 (or gamma_t = 0): no tangential force and no spin, the same
    # state as the frictionless model of R25
    base = W.packed_bed(dim=2, n=(12, 24))
    runs = []
    for mu, gt in ((0.0, 0.0), (0.0, 1e-6), (0.5, 0.0)):
        bed = O.OracleBed(base.with_(dem_mu=mu, dem_gamma_t=gt))
        bed.step(3)
        runs.append((*bed.particles(), bed.spin()))
    for P, V, sp in runs[1:]:
        np.testing.assert_array_equal(P, runs[0][0])
        np.testing.assert_array_equal(V, runs[0][1])
        assert not sp.any()


def _friction_bruteforce(P, v, wz, n, per, d, k, top_open=False):
    """All pairs and faces with friction (2D: spins about z)."""
    N, dim = P.shape
    r = 0.5 * d
    F = np.zeros((N, 2))
    T = np.zeros(N)

    def add(i, nrm, l, fn, vc):
        F[i] += fn * nrm
        vt = vc - (vc @ nrm) * nrm
        st = math.sqrt(vt @ vt)
        if fn > 0 and st > 0:
            ft = -min(k["gamma_t"] * st, k["mu_f"] * fn) * vt / st
            F[i] += ft
            arm = -l * nrm
            T[i] += arm[0] * ft[1] - arm[1] * ft[0]

    def wx(om, vec):                     # (0, 0, om) x vec in the plane
        return np.array([-om * vec[1], om * vec[0]])

    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            dx = P[i] - P[j]
            for a in range(dim):
                if per[a]:
                    dx[a] -= n[a] * round(dx[a] / n[a])
            dist = math.sqrt(dx @ dx)
            if dist >= d:
                continue
            nrm = dx / dist
            fn = max(k["kn"] * (d - dist) - k["eta"] * ((v[i] - v[j]) @ nrm), 0.0)
            l = 0.5 * dist
            add(i, nrm, l, fn, (v[i] - v[j]) - l * wx(wz[i] + wz[j], nrm))
        for a in range(dim):
            if per[a]:
                continue
            for side in (0, 1):
                l = P[i, a] if side == 0 else n[a] - P[i, a]
                if l >= r:
                    continue
                nrm = np.zeros(2)
                nrm[a] = 1.0 if side == 0 else -1.0
                fn = max(k["kn"] * (r - l) - k["eta_w"] * (v[i] @ nrm), 0.0)
                add(i, nrm, l, fn, v[i] - l * wx(wz[i], nrm))
    return F, T


@pytest.mark.parametrize("walls", [False, True])
def test_friction_forces_and_torques_match_all_pairs(walls):
    n = (7, 6)
    rng = np.random.default_rng(21)
    d = 0.7
    box = np.array(n, dtype=float)
    pos = W.rsa(2, box, [0.36] * 2, box - 0.36, (0, 0, 0) if walls else (1, 1, 1), 0.8 * d, 60, 9)
    vel = rng.normal(scale=2e-3, size=pos.shape)
    bc = (W.WALL,) * 6 if walls else (W.PERIODIC,) * 6
    w, mp, kn = _soft(dim=2, n=n, d_p=d, rho_s=50.0, e=0.6, contact_steps=12.0, bc=bc, pos=pos,
                      vel=vel, dem_mu=0.3, dem_gamma_t=2.0)
    bed = O.OracleBed(w)
    spin0 = rng.normal(scale=5e-3, size=len(pos))
    bed.set_spin(spin0)
    P0, v0 = bed.particles()
    k = bed.constants()
    bed.step(1)
    F, T = _friction_bruteforce(P0, v0, spin0, n, [not walls] * 2, d, k)
    fc = bed.particle_diag(O.P_FC)
    np.testing.assert_allclose(fc, F, rtol=0, atol=1e-12 * np.abs(F).max())
    np.testing.assert_allclose(bed.spin() - spin0, T / k["inertia"], rtol=0,
                               atol=1e-12 * np.abs(T / k["inertia"]).max())
    # both regimes occur: capped (Coulomb) and viscous contacts
    assert np.abs(T).max() > 0


# ------------------------------------------- sequential hard-sphere rule (R27)

def test_sequential_rule_newtons_cradle():
    # Three equal spheres in a row, all touching, the first moving into the
    # others (e = 1).  Resolving the contacts in order and re-checking the
    # approach passes the velocity down the row at once (0, 0, v); the
    # mutual-nearest rule (R14) resolves one binary collision per call, as
    # §2.2 describes binary collisions, and gets there in two.
    v = 0.01
    P = np.array([[2.0, 3.5], [2.0 + 0.99 * 0.5, 3.5], [2.0 + 2 * 0.99 * 0.5, 3.5]])
    V = np.array([[v, 0.0], [0.0, 0.0], [0.0, 0.0]])
    base = _bed(n=(8, 8), d_p=0.5, e=1.0, pos=np.zeros((0, 2)), vel=np.zeros((0, 2)))
    seq = O.OracleBed(types.SimpleNamespace(**{**vars(base), "collision_rule": 1}))
    seq.set_particles(P, V)
    seq.collide_particles()
    np.testing.assert_allclose(seq.particles()[1], [[0, 0], [0, 0], [v, 0]], atol=1e-17)
    match = O.OracleBed(base)
    match.set_particles(P, V)
    match.collide_particles()
    np.testing.assert_allclose(match.particles()[1], [[0, 0], [v, 0], [0, 0]], atol=1e-17)
    match.set_particles(P, match.particles()[1])
    match.collide_particles()
    np.testing.assert_allclose(match.particles()[1], [[0, 0], [0, 0], [v, 0]], atol=1e-17)


@pytest.mark.parametrize("dim", [2, 3])
def test_rules_agree_on_isolated_contacts(dim):
    # When no particle has more than one approaching contact the two rules
    # resolve the same pairs from the same velocities: identical results.
    rng = np.random.default_rng(4 + dim)
    n = (12, 12) if dim == 2 else (8, 8, 8)
    d = 0.4
    P, V = [], []
    for c in range(12):
        centre = (np.array([2 * (c % 4) + 1.5, 2 * (c // 4) + 1.5, 3.5]))[:dim]
        u = rng.normal(size=dim)
        u /= np.linalg.norm(u)
        P += [centre - 0.45 * d * u, centre + 0.45 * d * u]
        V += [0.01 * u + rng.normal(scale=1e-3, size=dim), -0.01 * u]
    P, V = np.array(P), np.array(V)
    base = _bed(dim=dim, n=n, d_p=d, e=0.7, pos=np.zeros((0, dim)), vel=np.zeros((0, dim)),
                bc=(W.WALL,) * 6)
    out = []
    for rule in (0, 1):
        bed = O.OracleBed(types.SimpleNamespace(**{**vars(base), "collision_rule": rule}))
        bed.set_particles(P, V)
        bed.collide_particles()
        out.append(bed.particles()[1])
        assert len(bed.pairs()) == 12
    np.testing.assert_array_equal(out[0], out[1])
    assert np.abs(out[0] - V).max() > 1e-3


@pytest.mark.parametrize("dim,n,N", [(2, (6, 7), 200), (3, (4, 5, 6), 200)])
def test_sequential_rule_keeps_momentum(dim, n, N):
    # a dense, overlapping state in a periodic box: each sequential binary
    # collision keeps momentum, so the total does
    P, v = _packed_state(dim, n, N, 0.9, 3)
    base = _bed(dim=dim, n=n, d_p=0.9, bc=(W.PERIODIC,) * 6, pos=np.zeros((0, dim)),
                vel=np.zeros((0, dim)))
    bed = O.OracleBed(types.SimpleNamespace(**{**vars(base), "collision_rule": 1}))
    bed.set_particles(P, v)
    bed.collide_particles()
    v1 = bed.particles()[1]
    assert np.abs(v1 - v).max() > 1e-3
    np.testing.assert_allclose(v1.sum(axis=0), v.sum(axis=0), rtol=0, atol=1e-12)


def test_sequential_rule_leaves_separating_contacts_alone():
    # R27 resolves a contact only if it approaches when its turn comes: a
    # touching pair moving apart keeps its velocities, and so does a pair
    # that an earlier collision in the order has turned around
    base = _bed(n=(8, 8), d_p=0.5, e=1.0, pos=np.zeros((0, 2)), vel=np.zeros((0, 2)))
    seq = O.OracleBed(types.SimpleNamespace(**{**vars(base), "collision_rule": 1}))
    P = np.array([[2.0, 3.5], [2.45, 3.5]])
    V = np.array([[-0.01, 0.0], [0.01, 0.0]])
    seq.set_particles(P, V)
    seq.collide_particles()
    np.testing.assert_array_equal(seq.particles()[1], V)
    # 0 and 1 approach, 1 and 2 touch while 2 runs ahead of 1 after the
    # first collision: (1, 2) is skipped
    P = np.array([[2.0, 3.5], [2.45, 3.5], [2.9, 3.5]])
    V = np.array([[0.01, 0.0], [0.0, 0.0], [0.02, 0.0]])
    seq.set_particles(P, V)
    seq.collide_particles()
    np.testing.assert_allclose(seq.particles()[1], [[0, 0], [0.01, 0], [0.02, 0]], atol=1e-17)


def _friction_bruteforce_3d(P, v, w, n, per, d, k):
    """All pairs and faces with friction in 3D (spins with three components)."""
    N = P.shape[0]
    r = 0.5 * d
    F = np.zeros((N, 3))
    T = np.zeros((N, 3))

    def add(i, nrm, l, fn, vc):
        F[i] += fn * nrm
        vt = vc - (vc @ nrm) * nrm
        st = math.sqrt(vt @ vt)
        if fn > 0 and st > 0:
            ft = -min(k["gamma_t"] * st, k["mu_f"] * fn) * vt / st
            F[i] += ft
            T[i] += np.cross(-l * nrm, ft)

    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            dx = P[i] - P[j]
            for a in range(3):
                if per[a]:
                    dx[a] -= n[a] * round(dx[a] / n[a])
            dist = math.sqrt(dx @ dx)
            if dist >= d:
                continue
            nrm = dx / dist
            fn = max(k["kn"] * (d - dist) - k["eta"] * ((v[i] - v[j]) @ nrm), 0.0)
            l = 0.5 * dist
            add(i, nrm, l, fn, (v[i] - v[j]) - l * np.cross(w[i] + w[j], nrm))
        for a in range(3):
            if per[a]:
                continue
            for side in (0, 1):
                l = P[i, a] if side == 0 else n[a] - P[i, a]
                if l >= r:
                    continue
                nrm = np.zeros(3)
                nrm[a] = 1.0 if side == 0 else -1.0
                fn = max(k["kn"] * (r - l) - k["eta_w"] * (v[i] @ nrm), 0.0)
                add(i, nrm, l, fn, v[i] - l * np.cross(w[i], nrm))
    return F, T


@pytest.mark.parametrize("walls", [False, True])
def test_friction_forces_and_torques_match_all_pairs_3d(walls):
    n = (4, 5, 4)
    rng = np.random.default_rng(31)
    d = 0.7
    box = np.array(n, dtype=float)
    pos = W.rsa(3, box, [0.36] * 3, box - 0.36, (0, 0, 0) if walls else (1, 1, 1), 0.8 * d, 90, 12)
    vel = rng.normal(scale=2e-3, size=pos.shape)
    bc = (W.WALL,) * 6 if walls else (W.PERIODIC,) * 6
    w, mp, kn = _soft(dim=3, n=n, d_p=d, rho_s=50.0, e=0.6, contact_steps=12.0, bc=bc, pos=pos,
                      vel=vel, dem_mu=0.3, dem_gamma_t=2.0)
    bed = O.OracleBed(w)
    spin0 = rng.normal(scale=5e-3, size=(len(pos), 3))
    bed.set_spin(spin0)
    P0, v0 = bed.particles()
    k = bed.constants()
    bed.step(1)
    F, T = _friction_bruteforce_3d(P0, v0, spin0, n, [not walls] * 3, d, k)
    np.testing.assert_allclose(bed.particle_diag(O.P_FC), F, rtol=0, atol=1e-12 * np.abs(F).max())
    np.testing.assert_allclose(bed.spin() - spin0, T / k["inertia"], rtol=0,
                               atol=1e-12 * np.abs(T / k["inertia"]).max())
    assert (np.abs(T).sum(axis=1) > 0).mean() > 0.3


def test_mutation_check_sample():
    # three planted mistakes from different parts of the oracle (the full
    # list, run by hand: python tests/mutation_check.py) are each caught
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, os.path.join(here, "mutation_check.py"), "-j", "3",
                        "-k", "omega_s sign", "-k", "cross3 sign", "-k", "tie to later"],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "3 of 3 caught" in r.stdout
