"""Seeded input generator: splitmix64 stream, RSA placement, Maxwellian."""
import numpy as np
import pytest

from paper_1303_2653_gb300 import workloads as W


def test_splitmix64_reference_outputs():
    # splitmix64 seeded with 0 (Steele, Lea and Flood 2014; reference outputs
    # of the public-domain C implementation)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = W.uniform_stream(0, 3)
    np.testing.assert_array_equal(u, [(z >> 11) * 2.0 ** -53 for z in want])


def test_rsa_non_overlapping_and_in_bounds():
    box, lo, hi, d = (1.0, 2.0), (0.05, 0.0), (0.95, 2.0), 0.02
    P = W.rsa(2, box, lo, hi, (0, 1), d, 1500, 42)
    assert P.shape == (1500, 2)
    assert (P[:, 0] >= lo[0]).all() and (P[:, 0] <= hi[0]).all()
    dx = P[:, None, 0] - P[None, :, 0]
    dy = P[:, None, 1] - P[None, :, 1]
    dy = np.where(dy > 1.0, dy - 2.0, np.where(dy < -1.0, dy + 2.0, dy))
    dist = np.sqrt(dx * dx + dy * dy) + np.eye(len(P)) * 10
    assert dist.min() >= d
    # seeded: identical on repeat
    np.testing.assert_array_equal(P, W.rsa(2, box, lo, hi, (0, 1), d, 1500, 42))


def test_maxwellian_moments():
    v = W.maxwellian(3, 200000, (0.0, 1.0, 0.0), 0.1, 9)
    np.testing.assert_allclose(v.mean(axis=0), [0.0, 1.0, 0.0], atol=2e-3)
    np.testing.assert_allclose(v.std(axis=0), 0.1, rtol=1e-2)


def test_riser_workload_shape():
    w = W.scaled_riser2d(nx=32, ny=64)
    assert w.n == (32, 64) and w.pos.shape == (w.n_particles, 2)
    area = w.n_particles * np.pi * (0.5 * w.d_p) ** 2 / (32 * 64 * w.h * w.h)
    assert abs(area - 0.05) < 1e-12


def test_soft_sphere_workload_helpers():
    import math
    from scipy.spatial.distance import pdist
    w = W.packed_bed(dim=2, n=(16, 24), gap=0.9, contact_steps=20.0)
    # centres at least gap d_p apart, inside the lower half, closed box
    assert pdist(w.pos).min() >= 0.9 * w.d_p * (1 - 1e-12)
    assert w.pos[:, 1].max() <= 12 * w.h and w.pos.min() >= 0.5 * w.d_p
    assert w.bc[:4] == (W.WALL,) * 4 and w.collision_model == 1
    # k_n makes an undamped pair contact (half a period, reduced mass m/2)
    # last the asked number of steps
    m_p = w.rho_s * math.pi * w.d_p ** 3 / 6.0
    t_c = math.pi * math.sqrt(0.5 * m_p / w.dem_kn)
    assert t_c / w.dt == pytest.approx(20.0, rel=1e-12)
    s = W.soft_spheres(W.riser2d(nx=32, ny=64, n_particles=500), contact_steps=8.0, e=0.5)
    assert s.collision_model == 1 and s.e == 0.5 and s.dem_kn == W.dem_stiffness(s, 8.0)
    f = W.with_friction(w, mu=0.3, gamma_frac=0.1)
    assert f.dem_mu == 0.3 and f.dem_gamma_t == pytest.approx(0.1 * m_p / w.dt, rel=1e-14)
    w3 = W.packed_bed(dim=3, n=(6, 6, 8), n_particles=2000)
    assert w3.pos.shape == (2000, 3) and pdist(w3.pos).min() >= 0.9 * w3.d_p * (1 - 1e-12)


def test_documented_workload_recipes():
    # the synthetic stand-ins for the paper's two simulations and the bench
    # beds carry the sizes and derived lattice quantities stated for them:
    # Table 1 (bubbling bed), Table 2 (riser), and the riser, bubbling and 3D
    # benches built on them
    import math
    from oracle import oracle as O
    area = lambda w, rows: w.n_particles * math.pi * (0.5 * w.d_p) ** 2 / (w.n[0] * rows * w.h ** 2)

    b = W.bubbling2d()
    k = O.units(b)
    assert (b.n, b.n_particles, b.h, b.dt, b.d_p, b.rho_s) == ((64, 128), 2000, 2e-3, 1e-4, 5e-4, 2500.0)
    assert k["tau"] == pytest.approx(0.50113, abs=1e-5)
    assert k["u0_y"] == pytest.approx(0.1885 * 1e-4 / 2e-3, rel=1e-3)
    jet = np.flatnonzero(b.inlet_u[:, 1] > 1.5 * b.inlet_u[:, 1].min())
    assert jet.tolist() == [30, 31, 32, 33]
    assert b.inlet_u[30, 1] == pytest.approx(5 * b.inlet_u[0, 1], rel=1e-12)

    r = W.riser2d()
    k = O.units(r)
    assert (r.n, r.n_particles, r.d_p, r.rho_s) == ((256, 2048), 200000, 54e-6, 930.0)
    assert area(r, 2048) == pytest.approx(0.05, rel=1e-12)
    assert r.h == pytest.approx(1.322e-4, rel=1e-3) and r.dt == pytest.approx(2.98e-6, rel=1e-3)
    assert k["tau"] == pytest.approx(0.50818, abs=1e-5) and k["u0_y"] == pytest.approx(0.0338)

    t1 = W.bubbling_table1()
    k = O.units(t1)
    assert (t1.n, t1.n_particles, t1.h, t1.dt) == ((25, 100), 15000, 2.7e-4, 1.35e-6)
    assert area(t1, 45) == pytest.approx(0.42, abs=2e-3)
    assert k["tau"] == pytest.approx(0.50089, abs=1e-5)

    t2 = W.cfb_riser2d()
    assert (t2.n, t2.n_particles) == ((60, 720), 123921)
    assert t2.dt == pytest.approx(6.0e-6, rel=1e-3)

    r3 = W.riser3d()
    k = O.units(r3)
    assert (r3.n, r3.n_particles) == ((256, 256, 1024), 4000000)
    vp = math.pi * r3.d_p ** 3 / 6
    assert r3.n_particles * vp / (math.prod(r3.n) * r3.h ** 3) == pytest.approx(0.03, rel=1e-12)
    assert r3.h == pytest.approx(5.47e-5, rel=1e-3) and r3.dt == pytest.approx(1.23e-6, abs=5e-9)
    assert k["tau"] == pytest.approx(0.5198, abs=1e-4)
