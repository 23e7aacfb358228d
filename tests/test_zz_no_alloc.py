"""The allocation-free cell binning entry point (lbdps_bin_sort_noalloc).

It serves callers that cannot allocate device memory while they run, for
example code being recorded into a CUDA graph or a host that owns a fixed
device-memory budget.  Here it is called through the C ABI on device buffers
that the test owns, and its cell list and sorted order are compared with
those of the handle-based path (lbdps_create / lbdps_step), bit for bit, on
calls made one after another.  The fixed scratch array keeps the previous
call's contents, so a second call with different positions checks that
nothing stale leaks into the result.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1303_2653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1303_2653_gb300 import build
    build.build_all()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _expected(bed, L):
    order = bed.particle_diag(L.PDIAG_ORDER).astype(np.int64)
    cells = bed.particle_diag(L.PDIAG_CELL).astype(np.int64)
    cs = np.r_[0, np.cumsum(np.bincount(cells, minlength=bed.ncell))]
    return cs, order


def _noalloc(bed, L, torch):
    P, _ = bed.particles()          # lattice units, id order
    dev = [torch.from_numpy(np.ascontiguousarray(P[:, a])).cuda() for a in range(bed.dim)]
    cs = torch.full((bed.ncell + 1,), -1, dtype=torch.int32, device="cuda")
    order = torch.full((max(bed.np, 1),), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    L.bin_sort_noalloc(bed.dim, bed.n, [t.data_ptr() for t in dev], cs.data_ptr(),
                       order.data_ptr(), bed.np, stream.cuda_stream)
    torch.cuda.synchronize()
    return cs.cpu().numpy().astype(np.int64), order.cpu().numpy()[: bed.np].astype(np.int64)


def test_noalloc_sort_matches_handle_sort_on_consecutive_calls():
    import torch
    from paper_1303_2653_gb300 import lbdps as L
    beds = [L.Bed(W.scaled_riser2d(nx=64, ny=128), storage=W.STORE_F32),
            L.Bed(W.scaled_riser3d(nx=12, ny=12, nz=24, n_particles=900, solid_fraction=0.08),
                  storage=W.STORE_F32)]
    calls = 0
    for bed in beds:
        for rep in range(2):
            cs_ref, order_ref = _expected(bed, L)
            cs, order = _noalloc(bed, L, torch)
            np.testing.assert_array_equal(cs, cs_ref)
            np.testing.assert_array_equal(order, order_ref)
            calls += 1
            bed.step(5)         # new positions for the next call
        bed.close()
    assert calls == 4


def _expected_clamped(P, n):
    """Cell list and (cell, id) order of positions clamped as the entry point
    documents: below 0 or NaN to the first cell of the axis, at or above n[a]
    to the last."""
    dim = P.shape[1]
    q = np.zeros(P.shape, dtype=np.int64)
    for a in range(dim):
        x = P[:, a]
        with np.errstate(invalid="ignore"):
            inside = (x >= 0) & (x < n[a])
            q[:, a] = np.where(inside, np.floor(np.where(inside, x, 0.0)), np.where(x >= n[a], n[a] - 1, 0))
    lin = q[:, 0] + n[0] * q[:, 1] + (n[0] * n[1] * q[:, 2] if dim == 3 else 0)
    ncell = int(np.prod(n))
    cs = np.r_[0, np.cumsum(np.bincount(lin, minlength=ncell))]
    return cs, np.lexsort((np.arange(len(lin)), lin))


def _call(L, torch, n, P):
    dim = len(n)
    ncell = int(np.prod(n))
    m = P.shape[0]
    dev = [torch.from_numpy(np.ascontiguousarray(P[:, a])).cuda() for a in range(dim)]
    cs = torch.full((ncell + 1,), -1, dtype=torch.int32, device="cuda")
    order = torch.full((max(m, 1),), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    L.bin_sort_noalloc(dim, n, [t.data_ptr() for t in dev], cs.data_ptr(), order.data_ptr(), m,
                       stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize()
    return (cs.cpu().numpy().astype(np.int64), order.cpu().numpy()[:m].astype(np.int64),
            a.elapsed_time(b))


def test_noalloc_clamps_positions_outside_the_lattice():
    # 100 x 130 cells: three full 4,096-cell scan tiles and a ragged fourth;
    # coordinates just below 0, at and above n[a], huge, infinite and NaN
    import torch
    from paper_1303_2653_gb300 import lbdps as L
    n = (100, 130)
    rng = np.random.default_rng(31)
    for rep in range(2):
        P = rng.uniform(0, 1, size=(20000, 2)) * np.array(n, dtype=float)
        odd = np.array([-1e-12, -0.5, -3e9, -1e300, -np.inf, np.nan, 0.0,
                        100.0, 130.0, 100.0 + 1e-9, 3e9, 1e300, np.inf, 99.99999999])
        for a in range(2):
            pick = rng.choice(len(P), size=300 * (rep + 1), replace=False)
            P[pick, a] = rng.choice(odd, size=len(pick))
        cs_ref, order_ref = _expected_clamped(P, n)
        cs, order, _ = _call(L, torch, n, P)
        np.testing.assert_array_equal(cs, cs_ref)
        np.testing.assert_array_equal(order, order_ref)


def test_noalloc_empty_and_three_dimensional_ragged():
    import torch
    from paper_1303_2653_gb300 import lbdps as L
    cs, order, _ = _call(L, torch, (7, 9, 11), np.zeros((0, 3)))
    np.testing.assert_array_equal(cs, np.zeros(7 * 9 * 11 + 1, dtype=np.int64))
    assert order.size == 0
    rng = np.random.default_rng(32)
    n = (17, 19, 23)
    P = rng.uniform(-0.5, 1.05, size=(5000, 3)) * np.array(n, dtype=float)
    cs_ref, order_ref = _expected_clamped(P, n)
    cs, order, _ = _call(L, torch, n, P)
    np.testing.assert_array_equal(cs, cs_ref)
    np.testing.assert_array_equal(order, order_ref)


def test_noalloc_largest_sizes_and_one_crowded_cell():
    # the limits: 2^20 cells and 2^20 particles, random; then every particle
    # in one cell (the order inside a cell comes from a radix sort, so this
    # costs the same as any other distribution)
    import torch
    from paper_1303_2653_gb300 import lbdps as L
    n = (1024, 1024)
    rng = np.random.default_rng(33)
    P = rng.uniform(0, 1, size=(1 << 20, 2)) * np.array(n, dtype=float)
    cs_ref, order_ref = _expected_clamped(P, n)
    cs, order, ms_random = _call(L, torch, n, P)
    np.testing.assert_array_equal(cs, cs_ref)
    np.testing.assert_array_equal(order, order_ref)
    P = np.full((1 << 20, 2), 517.25)
    cs, order, ms_crowded = _call(L, torch, n, P)
    c = 517 + 1024 * 517
    want = np.zeros(1024 * 1024 + 1, dtype=np.int64)
    want[c + 1:] = 1 << 20
    np.testing.assert_array_equal(cs, want)
    np.testing.assert_array_equal(order, np.arange(1 << 20))
    print(f"2^20 particles: random {ms_random:.3f} ms, all in one cell {ms_crowded:.3f} ms")
    assert ms_crowded < 50.0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1303_2653_gb300 import lbdps as L
    cs = torch.zeros(8, dtype=torch.int32, device="cuda")
    order = torch.zeros(8, dtype=torch.int32, device="cuda")
    pos = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LbdpsError) as ei:
        L.bin_sort_noalloc(2, (2048, 1024), [pos.data_ptr(), pos.data_ptr()], cs.data_ptr(),
                           order.data_ptr(), 8, torch.cuda.current_stream().cuda_stream)
    assert ei.value.code == L.ERR_CAPACITY
    assert "exceed" in str(ei.value)
