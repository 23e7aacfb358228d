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
