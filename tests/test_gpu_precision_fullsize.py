"""Reduced-precision storage and full-size beds against the oracle.

Reduced precision (FP16 x 2^10 and BF16 storage of f_i - w_i, FP32
arithmetic): from an identical state the node fields of one step come from
exactly representable inputs and keep the FP32 bounds; the stored
populations after the step must match the oracle within half an ulp of the
storage format at their magnitude plus the FP32 bound.

Full size: the riser 256 x 2048 with 200,000 particles (the configuration
bench.py times, same launch path) takes the one-step parity check in full;
the D3Q19 riser 256 x 256 x 1024 with 4,000,000 particles (too large for the
oracle) is checked through properties that hold at any size: bit-exact cell
sort against numpy, exact particle count, gas mass conserved to the FP32
rounding of the stored deviations, finite state.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_2653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1303_2653_gb300 import build
    build.build_all()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _lb():
    from paper_1303_2653_gb300 import lbdps
    return lbdps


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def _half_ulp(x, storage):
    """Half an ulp of the stored deviation x (FP16 of x * 2^10, or BF16)."""
    x = np.abs(x)
    if storage == W.STORE_F16:
        s = x * 1024.0
        e = np.floor(np.log2(np.maximum(s, 2.0 ** -14)))
        return 0.5 * 2.0 ** (e - 10) / 1024.0
    e = np.floor(np.log2(np.maximum(x, 2.0 ** -126)))
    return 0.5 * 2.0 ** (e - 7)


@pytest.mark.parametrize("storage", [W.STORE_F16, W.STORE_BF16])
def test_reduced_precision_one_step(storage):
    L = _lb()
    w = W.scaled_riser2d(nx=48, ny=96, seed=31)
    bed = L.Bed(w, storage=storage, diagnostics=True)
    ob = O.OracleBed(w)
    f0 = bed.populations()
    ob.set_populations(f0)
    P, v = bed.particles()
    ob.set_particles(P, v)
    bed.step(1)
    ob.step(1)
    g = bed.fields(L.FIELD_RHO | L.FIELD_U | L.FIELD_FPG | L.FIELD_BETA)
    assert np.abs(g["rho"] - ob.field(O.F_RHO)).max() <= 2e-6
    assert _rel(g["u"], ob.field(O.F_U)) <= 2e-6
    assert _rel(g["fpg"], ob.field(O.F_FPG)) <= 1e-5
    assert _rel(g["beta"], ob.field(O.F_BETA)) <= 1e-5
    # stored populations: rounding of the deviation within half an ulp of the format
    fg, fo = bed.populations(), ob.populations()
    w_i = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None]
    dev_o = fo - w_i
    bound = _half_ulp(dev_o, storage) * 1.01 + 2e-6 * np.abs(dev_o).max()
    assert np.all(np.abs(fg - fo) <= bound)
    # and the rounding is really at the storage precision (not FP32)
    assert np.abs(fg - fo).max() > 1e-3 * _half_ulp(np.abs(dev_o).max(), storage)
    bed.close()


def test_riser_full_size_one_step_parity():
    """256 x 2048, 200,000 particles, FP32 storage, graph launch as in bench.py."""
    L = _lb()
    w = W.riser2d()
    bed = L.Bed(w, storage=W.STORE_F32, diagnostics=True)
    ob = O.OracleBed(w)
    ob.set_populations(bed.populations())
    P0, v0 = bed.particles()
    ob.set_particles(P0, v0)
    order = bed.particle_diag(L.PDIAG_ORDER).astype(np.int64)
    ids, _ = ob.sorted_ids()
    np.testing.assert_array_equal(order, ids)
    bed.step(1)
    ob.step(1)
    g = bed.fields(L.FIELD_RHO | L.FIELD_U | L.FIELD_FPG | L.FIELD_BETA | L.FIELD_NTOT)
    np.testing.assert_array_equal(g["ntot"], ob.field(O.F_NTOT))
    assert _rel(g["u"], ob.field(O.F_U)) <= 2e-6
    assert np.abs(g["rho"] - ob.field(O.F_RHO)).max() <= 2e-6
    assert _rel(g["fpg"], ob.field(O.F_FPG)) <= 1e-5
    assert _rel(g["beta"], ob.field(O.F_BETA)) <= 1e-5
    Pg, vg = bed.particles()
    Po, vo = ob.particles()
    # well-conditioned Eq. 28 cells (see test_gpu_parity): velocities within 1e-5
    S, A = ob.field(O.F_SUM_PRE), ob.field(O.F_SUM_ABS_PRE)
    with np.errstate(divide="ignore", invalid="ignore"):
        kappa = np.where(A > 0, np.where(np.abs(S) > 0, A / np.abs(S), np.inf), 1.0).max(axis=1)
    c0 = np.floor(P0).astype(np.int64)
    cell0 = c0[:, 0] + w.n[0] * c0[:, 1]
    good = kappa[cell0] < 1e3
    assert good.mean() > 0.95
    assert _rel(vg[good], vo[good]) <= 1e-5
    assert np.abs(Pg[good] - Po[good]).max() <= 1e-6
    # cells of the new sort: equal except where the two positions straddle a face
    cg = bed.particle_diag(L.PDIAG_CELL).astype(np.int64)
    co = ob.particle_diag(O.P_CELL).astype(np.int64)
    mism = cg != co
    if mism.any():
        frac = np.abs(Po[mism] - np.round(Po[mism]))
        assert frac.min(axis=1).max() < 1e-4
    bed.close()


def test_riser3d_full_size_properties():
    """256 x 256 x 1024 D3Q19, 4,000,000 particles, FP32 (about 13 GB on the device)."""
    L = _lb()
    w = W.riser3d()
    bed = L.Bed(w, storage=W.STORE_F32, torch_memory=False)
    m0 = bed.stats()["mass"]
    bed.step(3)
    st = bed.stats()
    assert st["health"] == 0
    # mass: each step rounds every stored deviation to FP32 (|dev| < 0.05)
    assert abs(st["mass"] - m0) <= 3 * 19 * w.ncell * 0.05 * 2.0 ** -24 * 4
    P, v = bed.particles()
    assert P.shape == (4000000, 3) and np.isfinite(P).all() and np.isfinite(v).all()
    cell = np.floor(P).astype(np.int64)
    lin = cell[:, 0] + 256 * (cell[:, 1] + 256 * cell[:, 2])
    order = bed.particle_diag(L.PDIAG_ORDER).astype(np.int64)
    np.testing.assert_array_equal(order, np.lexsort((np.arange(len(lin)), lin)))
    bed.close()
