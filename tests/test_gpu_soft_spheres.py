"""GPU vs oracle: soft-sphere contacts (the DEM option for dense beds).

Both sides start from the same state (the GPU bed's populations and
particles loaded into the oracle).  The contact forces of a step come from
that common state, so they are compared per particle: FP64 to 1e-11 and FP32
to 1e-5 of the largest force (the overlap is formed from an exact FP64
difference, so FP32 keeps its relative precision; normals, approach speeds
and up to a dozen contacts per particle are summed in FP32).  The integrated
state then follows the drag bounds of the hard-sphere parity tests.
"""
import math
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from oracle import oracle as O                      # noqa: E402
from paper_1303_2653_gb300 import workloads as W    # noqa: E402
from test_gpu_parity import TOL_DERIVED, _compare_step, _pair, _particle_compare   # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1303_2653_gb300 import build
    build.build_all()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _lb():
    from paper_1303_2653_gb300 import lbdps as L
    return L


def _packed(name, storage):
    if name == "packed2d":
        return W.packed_bed(dim=2, n=(24, 48), storage=storage)
    return W.packed_bed(dim=3, n=(8, 8, 12), storage=storage, seed=W.SEED_BASE + 8)


def _lattice_pair(e, contact_steps, storage, v=1e-3):
    """Head-on pair in a periodic 16 x 8 box, h = dt = rho_g = 1 (lattice
    units), heavy particles so that the gas barely acts on them."""
    d, rho_s = 0.5, 1e6
    mp = rho_s * math.pi * d ** 3 / 6.0
    kn = 0.5 * mp * (math.pi / contact_steps) ** 2
    # the gap closes in 21.3 steps: no step ends near the contact threshold,
    # so that both sides start the contact in the same step
    P = np.array([[8 - 0.25 - 0.0213, 4.3], [8 + 0.25 + 0.0213, 4.3]])
    V = np.array([[v, 0.0], [-v, 0.0]])
    return W.Workload(name="pair", dim=2, n=(16, 8), bc=(W.PERIODIC,) * 6, h=1.0, dt=1.0, d_p=d,
                      rho_s=rho_s, e=e, pos=P, vel=V, rho_g=1.0, mu_g=0.1, storage=storage,
                      collision_model=1, dem_kn=kn)


def test_soft_constants_match_oracle():
    L = _lb()
    w = _packed("packed2d", W.STORE_F32)
    bed, ob = _pair(w, W.STORE_F32)
    g, o = bed.constants(), ob.constants()
    for k in ("kn", "eta", "eta_w", "mp", "d", "r"):
        assert g[k] == pytest.approx(o[k], rel=1e-15), k
    assert g["kn"] > 0 and g["eta"] > 0
    bed.close()


@pytest.mark.parametrize("name", ["packed2d", "packed3d"])
@pytest.mark.parametrize("storage", [W.STORE_F64, W.STORE_F32])
def test_soft_one_step_parity(name, storage):
    L = _lb()
    w = _packed(name, storage)
    bed, ob = _pair(w, storage)
    Pg0, _ = bed.particles()
    n = w.n
    c0 = np.floor(Pg0).astype(np.int64)
    cell0 = c0[:, 0] + n[0] * c0[:, 1] + (n[0] * n[1] * c0[:, 2] if w.dim == 3 else 0)
    _compare_step(bed, ob, storage)
    fc_g = bed.particle_diag(L.PDIAG_FC)
    fc_o = ob.particle_diag(O.P_FC)
    in_contact = np.abs(fc_o).sum(axis=1) > 0
    assert in_contact.mean() > 0.2
    tol_f = 1e-11 if storage == W.STORE_F64 else 1e-5
    fmax = np.abs(fc_o).max()
    err = np.abs(fc_g - fc_o).max(axis=1) / fmax
    worst = int(np.argmax(err))
    assert err.max() <= tol_f, (worst, fc_g[worst].tolist(), fc_o[worst].tolist())
    np.testing.assert_array_equal(np.abs(fc_g).sum(axis=1) > 0, in_contact)
    # integrated state: the drag bound of the hard-sphere parity tests
    # (amplified where the Eq. 28 rescale is ill-conditioned) plus the
    # contact-force bound, each divided by m_p
    Pg, vg, Po, vo, fd_g, fd_o, kappa_cell = _particle_compare(bed, ob, storage)
    kappa = kappa_cell[cell0]
    good = kappa < 1e3
    assert good.mean() > 0.9
    tol_d = TOL_DERIVED[storage]
    amp = np.maximum(1.0, kappa / 100.0)[good][:, None]
    mp = ob.constants()["mp"]
    bound = tol_d * np.abs(fd_o).max() * amp / mp + tol_f * fmax / mp
    vmax = np.abs(vo).max()
    assert np.all(np.abs(vg[good] - vo[good]) <= bound + tol_d * vmax * amp)
    assert np.all(np.abs(Pg[good] - Po[good]) <= 4 * (bound + tol_d * vmax * amp) + 1e-13)
    assert bed.check_guards() == 0
    bed.close()


def test_soft_twenty_steps_fp64():
    # The gas here is nearly at rest (|u| ~ 1e-7) while the populations are
    # O(1), so u carries an absolute rounding floor of a few 1e-16 per step
    # on top of the relative bound
    L = _lb()
    w = _packed("packed2d", W.STORE_F64)
    bed, ob = _pair(w, W.STORE_F64)
    bed.step(20)
    ob.step(20)
    gf = bed.fields(L.FIELD_RHO | L.FIELD_U)
    u_o = ob.field(O.F_U)
    assert np.abs(gf["u"] - u_o).max() <= 1e-12 * np.abs(u_o).max() + 20 * 1e-15
    assert np.abs(gf["rho"] - ob.field(O.F_RHO)).max() <= 20 * 1e-15
    Pg, vg = bed.particles()
    Po, vo = ob.particles()
    assert np.abs(vg - vo).max() <= 1e-9 * np.abs(vo).max()
    assert np.abs(Pg - Po).max() <= 1e-10
    bed.close()


@pytest.mark.parametrize("storage", [W.STORE_F64, W.STORE_F32])
@pytest.mark.parametrize("e", [0.9, 0.5])
def test_soft_pair_collision_on_gpu(storage, e):
    # the whole contact of a head-on pair, step by step against the oracle
    L = _lb()
    w = _lattice_pair(e, 40.0, storage)
    bed = L.Bed(w, storage=storage)
    ob = O.OracleBed(w)
    ob.set_populations(bed.populations())
    vmax = 2e-3
    for _ in range(12):
        bed.step(10)
        ob.step(10)
        Pg, vg = bed.particles()
        Po, vo = ob.particles()
        tol = 1e-12 if storage == W.STORE_F64 else 2e-5
        assert np.abs(vg - vo).max() <= tol * vmax
        assert np.abs(Pg - Po).max() <= 1e-12 + 10 * tol * vmax * 10
    # separated again with the oracle's restitution
    e_g = (vg[1, 0] - vg[0, 0]) / vmax
    e_o = (vo[1, 0] - vo[0, 0]) / vmax
    assert e_g == pytest.approx(e_o, abs=1e-4)
    assert Pg[1, 0] - Pg[0, 0] > 0.5
    bed.close()


@pytest.mark.parametrize("storage", [W.STORE_F64, W.STORE_F32])
def test_soft_sphere_rests_on_the_floor_on_gpu(storage):
    # overlap on the floor = m_p g_eff / k_n once the bounce has died out
    L = _lb()
    g = 1e-5
    d, rho_s = 0.5, 1e6
    mp = rho_s * math.pi * d ** 3 / 6.0
    kn = 0.5 * mp * (math.pi / 40.0) ** 2
    w = W.Workload(name="floor", dim=2, n=(8, 8), bc=(W.WALL,) * 6, h=1.0, dt=1.0, d_p=d,
                   rho_s=rho_s, e=0.3, pos=np.array([[3.4, 0.5]]), vel=np.zeros((1, 2)),
                   rho_g=1.0, mu_g=0.1, g=(0.0, -g, 0.0), storage=storage, collision_model=1,
                   dem_kn=kn)
    bed = L.Bed(w, storage=storage)
    bed.step(3000)
    P, v = bed.particles()
    g_eff = (1.0 - 1.0 / rho_s) * g
    tol = 1e-9 if storage == W.STORE_F64 else 2e-5
    assert P[0, 1] == pytest.approx(0.25 - mp * g_eff / kn, rel=tol)
    bed.close()


def test_soft_chunked_steps_equal_single_steps():
    L = _lb()
    w = _packed("packed2d", W.STORE_F32)
    a = L.Bed(w, check_every=24)
    b = L.Bed(w, use_graph=False)
    a.step(37)
    for _ in range(37):
        b.step(1)
    np.testing.assert_array_equal(a.populations(), b.populations())
    Pa, va = a.particles()
    Pb, vb = b.particles()
    np.testing.assert_array_equal(Pa, Pb)
    np.testing.assert_array_equal(va, vb)
    assert a.check_guards() == 0 and b.check_guards() == 0
    a.close()
    b.close()


def test_soft_profiled_classes_and_outlet():
    # the profiled step reports the contact kernel under the particle class;
    # with the solids loop closed, a particle leaves through the outlet
    L = _lb()
    w = W.cfb_riser2d(nx=16, ny=40, n_particles=60, seed=9, storage=W.STORE_F32, cs_smag=0.0)
    r = 0.5 * w.d_p / w.h
    P = np.array([[4.5, w.n[1] - 0.5 * r], [8.5, 0.5 * r]])
    v = np.array([[0.0, 0.08], [0.0, -0.01]])
    w = W.soft_spheres(w, contact_steps=20.0).with_(pos=P * w.h, vel=v * w.h / w.dt)
    bed = L.Bed(w, diagnostics=True)
    ob = O.OracleBed(w)
    ob.set_populations(bed.populations())
    ms = list(bed.step_profiled(1).values())
    ob.step(1)
    assert len(ms) == 4 and ms[3] > 0
    fc = bed.particle_diag(L.PDIAG_FC)
    np.testing.assert_allclose(fc, ob.particle_diag(O.P_FC), rtol=1e-5, atol=0)
    assert fc[0, 1] == 0.0 and fc[1, 1] > 0.0
    assert bed.stats()["solids_out"] == 1
    bed.close()


def test_soft_create_rules():
    L = _lb()
    w = _packed("packed2d", W.STORE_F32)
    # soft spheres may start in contact; hard spheres may not
    P = w.pos.copy()
    P[1] = P[0] + np.array([0.5 * w.d_p, 0.0])
    L.Bed(w.with_(pos=P)).close()
    with pytest.raises(L.LbdpsError):
        L.Bed(w.with_(pos=P, collision_model=0))
    for bad in (dict(dem_kn=0.0), dict(e=0.0), dict(collision_model=2),
                dict(dem_kn=W.dem_stiffness(w, 3.0))):
        with pytest.raises(L.LbdpsError) as ei:
            L.Bed(w.with_(**bad))
        assert ei.value.code == L.ERR_INVALID
    # 4 steps per contact is the stiffest accepted
    L.Bed(w.with_(dem_kn=W.dem_stiffness(w, 4.01))).close()
    # the contact diagnostic needs the soft model
    hb = L.Bed(W.scaled_riser2d(nx=32, ny=64), diagnostics=True)
    with pytest.raises(L.LbdpsError):
        hb.particle_diag(L.PDIAG_FC)
    hb.close()


def _wide_periodic(collision_model, storage, nx=2050):
    """Pairs straddling the periodic x face of a 2050-cell-wide box (lattice
    units): the x separation of a pair across the face is formed from cell
    offsets of nx - 1, where an FP32 intermediate of that size would round
    by about 1e-4."""
    rng = np.random.default_rng(3)
    d = 0.5
    P, V = [], []
    for k in range(12):
        y = 0.5 + k * 0.9
        gap = rng.uniform(0.38, 0.52)          # some overlap, some do not touch
        xa = rng.uniform(0.0, gap)
        P += [[xa, y], [nx - (gap - xa), y]]
        V += [[-1e-3, 0.0], [1e-3, 0.0]]       # approaching across the face
    P, V = np.array(P), np.array(V)
    return W.Workload(name="wide", dim=2, n=(nx, 12), bc=(W.PERIODIC,) * 6, h=1.0, dt=1.0, d_p=d,
                      rho_s=1e6, e=0.8, pos=P, vel=V, rho_g=1.0, mu_g=0.1, storage=storage,
                      collision_model=collision_model,
                      dem_kn=0.5 * 1e6 * math.pi * d ** 3 / 6.0 * (math.pi / 30.0) ** 2)


@pytest.mark.parametrize("storage", [W.STORE_F64, W.STORE_F32])
def test_contacts_across_a_wide_periodic_face(storage):
    L = _lb()
    # soft spheres: forces against the oracle
    w = _wide_periodic(1, storage)
    bed = L.Bed(w, storage=storage, diagnostics=True)
    ob = O.OracleBed(w)
    ob.set_populations(bed.populations())
    bed.step(1)
    ob.step(1)
    fo = ob.particle_diag(O.P_FC)
    fg = bed.particle_diag(L.PDIAG_FC)
    assert (np.abs(fo).sum(axis=1) > 0).sum() >= 8
    tol = 1e-11 if storage == W.STORE_F64 else 1e-5
    assert np.abs(fg - fo).max() <= tol * np.abs(fo).max()
    bed.close()
    # hard spheres: the same contact pairs as the oracle
    w = _wide_periodic(0, storage)
    touching = np.abs(w.pos[0::2, 0] + w.n[0] - w.pos[1::2, 0]) < w.d_p
    w = w.with_(pos=np.concatenate([w.pos[0::2][~touching], w.pos[1::2][~touching]]),
                vel=np.concatenate([w.vel[0::2][~touching], w.vel[1::2][~touching]]))
    bed = L.Bed(w, storage=storage)
    P, v = bed.particles()
    # bring each pair into contact across the face, then detect
    m = len(P) // 2
    P[m:, 0] = w.n[0] - (0.45 - P[:m, 0])
    bed.set_particles(P, v)
    ob = O.OracleBed(w)
    ob.set_particles(P, v)
    ob.collide_particles()
    pg = bed.collide_particles()
    np.testing.assert_array_equal(pg, ob.pairs())
    assert len(pg) == m
    bed.close()


# ------------------------------------------------------------------ friction

def _fric_pair(w, storage, seed=4):
    """GPU bed and oracle from the same state, with the same random spins."""
    bed, ob = _pair(w, storage)
    rng = np.random.default_rng(seed)
    nc = 1 if w.dim == 2 else 3
    spin = rng.normal(scale=2e-3, size=(len(w.pos), nc)).reshape(-1)
    bed.set_spin(spin)
    ob.set_spin(bed.spin())
    return bed, ob


def test_friction_constants_match_oracle():
    w = W.with_friction(_packed("packed2d", W.STORE_F32))
    bed, ob = _pair(w, W.STORE_F32)
    g, o = bed.constants(), ob.constants()
    for k in ("mu_f", "gamma_t", "inertia"):
        assert g[k] == pytest.approx(o[k], rel=1e-15), k
    assert g["gamma_t"] > 0
    bed.close()


@pytest.mark.parametrize("name", ["packed2d", "packed3d"])
@pytest.mark.parametrize("storage", [W.STORE_F64, W.STORE_F32])
def test_friction_one_step_parity(name, storage):
    L = _lb()
    w = W.with_friction(_packed(name, storage))
    bed, ob = _fric_pair(w, storage)
    s0 = bed.spin()
    bed.step(1)
    ob.step(1)
    tol = 1e-11 if storage == W.STORE_F64 else 1e-5
    fc_g, fc_o = bed.particle_diag(L.PDIAG_FC), ob.particle_diag(O.P_FC)
    assert np.abs(fc_g - fc_o).max() <= tol * np.abs(fc_o).max()
    ds_g, ds_o = bed.spin() - s0, ob.spin() - s0
    assert np.abs(ds_o).max() > 0
    assert np.abs(ds_g - ds_o).max() <= tol * np.abs(ds_o).max()
    Pg, vg = bed.particles()
    Po, vo = ob.particles()
    assert np.abs(vg - vo).max() <= 20 * tol * np.abs(vo).max()
    assert bed.check_guards() == 0
    bed.close()


def test_friction_ten_steps_fp64():
    w = W.with_friction(_packed("packed2d", W.STORE_F64))
    bed, ob = _fric_pair(w, W.STORE_F64)
    bed.step(10)
    ob.step(10)
    Pg, vg = bed.particles()
    Po, vo = ob.particles()
    assert np.abs(vg - vo).max() <= 1e-9 * np.abs(vo).max()
    assert np.abs(Pg - Po).max() <= 1e-10
    assert np.abs(bed.spin() - ob.spin()).max() <= 1e-9 * np.abs(ob.spin()).max()
    bed.close()


@pytest.mark.parametrize("storage", [W.STORE_F64, W.STORE_F32])
@pytest.mark.parametrize("dim", [2, 3])
def test_friction_rolling_on_gpu(storage, dim):
    # sliding turns into rolling at v0 / (1 + I / (m l^2))
    L = _lb()
    g, v0, d, rho_s, steps = 1e-5, 1e-3, 0.5, 1e9, 40.0
    mp = rho_s * math.pi * d ** 3 / 6.0
    kn = 0.5 * mp * (math.pi / steps) ** 2
    l = 0.25 - mp * (1.0 - 1.0 / rho_s) * g / kn
    n = (16, 8) if dim == 2 else (16, 6, 8)
    P = np.full((1, dim), 3.0)
    P[0, -1] = l
    V = np.zeros((1, dim))
    V[0, 0] = v0
    grav = (0.0, -g, 0.0) if dim == 2 else (0.0, 0.0, -g)
    w = W.Workload(name="roll", dim=dim, n=n, bc=(W.WALL,) * 6, h=1.0, dt=1.0, d_p=d, rho_s=rho_s,
                   e=0.3, pos=P, vel=V, rho_g=1.0, mu_g=0.1, g=grav, storage=storage,
                   collision_model=1, dem_kn=kn, dem_mu=0.5, dem_gamma_t=0.08 * mp)
    bed = L.Bed(w, storage=storage)
    bed.step(1500)
    Pn, Vn = bed.particles()
    inertia = bed.constants()["inertia"]
    tol = 1e-6 if storage == W.STORE_F64 else 1e-4
    assert Vn[0, 0] == pytest.approx(v0 / (1.0 + inertia / (mp * l * l)), rel=tol)
    spin = bed.spin()
    om = spin[0] if dim == 2 else spin[0, 1]
    # rolling along +x on a floor below: w_z = -v / l in 2D, w_y = v / l in 3D
    assert om == pytest.approx((-1.0 if dim == 2 else 1.0) * Vn[0, 0] / l, rel=tol)
    bed.close()


def test_friction_spins_checkpoint_and_reset():
    L = _lb()
    w = W.with_friction(_packed("packed2d", W.STORE_F32))
    a = L.Bed(w)
    a.step(20)
    blob = a.save()
    a.step(15)
    b = L.Bed(w)
    b.load(blob)
    b.step(15)
    np.testing.assert_array_equal(a.spin(), b.spin())
    np.testing.assert_array_equal(a.particles()[1], b.particles()[1])
    assert np.abs(a.spin()).max() > 0
    P, v = a.particles()
    a.set_particles(P, v)
    assert not a.spin().any()
    a.close()
    b.close()
    # spins only exist with friction
    c = L.Bed(_packed("packed2d", W.STORE_F32))
    assert not c.spin().any()
    with pytest.raises(L.LbdpsError):
        c.set_spin(np.ones(c.np))
    c.close()


def test_friction_create_rules():
    L = _lb()
    w = W.with_friction(_packed("packed2d", W.STORE_F32))
    m_p = w.rho_s * math.pi * w.d_p ** 3 / 6.0
    for bad in (dict(dem_mu=-0.1), dict(dem_gamma_t=0.3 * m_p / w.dt),
                dict(collision_model=0, pos=W.scaled_riser2d(nx=32, ny=64).pos,
                     vel=np.zeros_like(W.scaled_riser2d(nx=32, ny=64).pos))):
        with pytest.raises(L.LbdpsError) as ei:
            L.Bed(w.with_(**bad))
        assert ei.value.code == L.ERR_INVALID
    L.Bed(w.with_(dem_gamma_t=0.25 * m_p / w.dt * (1 - 1e-9))).close()


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_soft_long_run_statistics(mu):
    # 2,000 steps of the dense bed in FP32 on the GPU against the FP64
    # oracle from the same start: trajectories part ways (chaos), bed
    # statistics do not (within 1 % for the mean voidage, 5 % for the mean
    # particle speed, 0.05 cells for the mean particle height)
    L = _lb()
    w = W.packed_bed(dim=2, n=(24, 48), storage=W.STORE_F32)
    if mu > 0:
        w = W.with_friction(w, mu=mu)
    bed, ob = _pair(w, W.STORE_F32)
    bed.step(2000)
    ob.step(2000)
    sg, so = bed.stats(), ob.stats()
    assert sg["mean_eps_g"] == pytest.approx(so["mean_eps_g"], rel=1e-2)
    Pg, vg = bed.particles()
    Po, vo = ob.particles()
    assert np.abs(vg).mean() == pytest.approx(np.abs(vo).mean(), rel=5e-2)
    assert abs(Pg[:, 1].mean() - Po[:, 1].mean()) < 0.05
    assert sg["mass"] == pytest.approx(so["mass"], rel=1e-6)
    bed.close()


def test_packed_cell_is_reported_not_failed():
    # more particle centres in a cell than can be there without overlaps
    # (the close-packing count of the cell grown by one diameter; possible
    # with overlapping soft spheres, and what piled-up hard spheres reach in
    # a settled dense bed) sets health bit 8; stepping with check_every
    # carries on, since the state is valid
    L = _lb()
    w = W.packed_bed(dim=2, n=(12, 12), n_particles=60, storage=W.STORE_F32)
    rng = np.random.default_rng(8)
    P = w.pos.copy()
    P[:50] = (np.array([5.0, 5.0]) + rng.uniform(0.05, 0.95, size=(50, 2))) * w.h
    w = w.with_(pos=P)
    dl = w.d_p / w.h
    cap = math.pi / (2 * math.sqrt(3)) * (1 + dl) ** 2 / (math.pi * (0.5 * dl) ** 2)
    assert 50 > math.ceil(cap)
    bed = L.Bed(w, check_every=4)
    bed.step(8)
    assert bed.stats()["health"] & 8
    assert not bed.stats()["health"] & 3
    bed.close()
    # a bed within close packing does not set it
    ok = L.Bed(W.packed_bed(dim=2, n=(24, 48), storage=W.STORE_F32), check_every=4)
    ok.step(8)
    assert ok.stats()["health"] == 0
    ok.close()
