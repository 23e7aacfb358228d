"""Multi-rank logic of bench.py on CPU: world size 2 over gloo.

bench.py runs one independent bed per rank (replicas, weak scaling): the
job time is the maximum over ranks and the value counts the cell updates of
every rank.  The reference arm runs on rank 0 only.
"""
import io
import os
import socket
import sys
import contextlib

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) * 10 ms: the job time is the slowest rank's
    t = bench.max_over_ranks((rank + 1) * 10.0, dist, device="cpu")
    value = bench.whole_job_mlups(world, 1000, 50, t / 1e3)
    # the reference arm prints on rank 0 only; other ranks return at once
    buf = io.StringIO()
    if rank != 0:
        class A:
            pass
        with contextlib.redirect_stdout(buf):
            bench.reference_main(A(), rank, world)
    out.put((rank, t, value, buf.getvalue()))
    dist.destroy_process_group()


def test_two_ranks_take_the_max_time_and_count_all_cells():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value, printed in res:
        assert t == 20.0
        assert value == pytest.approx(2 * 1000 * 50 / 0.020 / 1e6)
        assert printed == ""


def test_oracle_sample_is_a_slab_of_large_beds():
    # the CPU baseline times the oracle on the full bed when it is small and
    # on a slab with the full cross section and the same solid fraction
    import bench
    from paper_1303_2653_gb300 import workloads as W
    small = W.scaled_riser2d(nx=32, ny=64)
    s, what = bench.oracle_sample(small)
    assert what == "the full bed" and s.n == small.n and s.storage == W.STORE_F64
    big = W.scaled_riser3d(nx=32, ny=32, nz=256)
    s, what = bench.oracle_sample(big, max_cells=50_000)
    assert s.n == (32, 32, 48) and "slab" in what
    assert s.bc == big.bc and s.storage == W.STORE_F64
    assert abs(s.n_particles / s.ncell - big.n_particles / big.ncell) <= 1.0 / s.ncell
    assert s.h == pytest.approx(big.h, rel=0.02) and s.d_p == big.d_p


def test_drag_step_bytes_and_kernel_roofline():
    # per particle: cell key 4 + P, v, off read (2D FP32: 16 + 8 + 8) and
    # written + new key 4 + histogram count 4; per cell: rho, u_act[2],
    # F_p->g[2], beta, 1 - eps (7 x 4) + the cell-list offset 4
    import bench
    from paper_1303_2653_gb300 import workloads as W
    w = W.scaled_riser2d(nx=32, ny=64)
    total, per_cell, per_particle = bench.drag_step_bytes(w, "f32")
    assert (per_cell, per_particle) == (32, 76)
    assert total == 32 * 32 * 64 + 76 * w.n_particles
    w3 = W.scaled_riser3d(nx=8, ny=8, nz=16)
    assert bench.drag_step_bytes(w3, "f64")[1:] == (9 * 8 + 4, 4 + 2 * (24 + 48) + 8)
    r = bench.kernel_roofline(2e9, 1.0, 4000.0)     # 2 GB in 1 ms: 2,000 GB/s
    assert r["achieved"] == pytest.approx(2000.0) and r["frac"] == pytest.approx(0.5)
    assert bench.kernel_roofline(2e9, 0.0, 4000.0) is None


def test_step_byte_models_match_the_planned_figures():
    # B_ideal = N_cells (2 Q s_f + c_cell) + N_p 4 s_p, c_cell = the 4-byte
    # cell-list offset + rho, u and F_p->g read by the drag; the planned
    # figures per configuration: 1.80 MB (bubbling 64 x 128, FP64, 2,000
    # particles), 69.5 MB (riser 256 x 2048, 200,000), 50.7 MB (the same in
    # 16-bit storage), 12.92 GB (3D riser 256 x 256 x 1024, 4,000,000)
    import types
    import bench

    def shape(dim, n, n_particles):
        ncell = 1
        for v in n:
            ncell *= v
        return types.SimpleNamespace(dim=dim, n=n, ncell=ncell, n_particles=n_particles)

    bubbling = shape(2, (64, 128), 2000)
    riser = shape(2, (256, 2048), 200000)
    riser3d = shape(3, (256, 256, 1024), 4000000)
    assert bench.whole_step_bytes(bubbling, "f64") == pytest.approx(1.80e6, abs=0.005e6)
    assert bench.whole_step_bytes(riser, "f32") == pytest.approx(69.5e6, abs=0.05e6)
    assert bench.whole_step_bytes(riser, "f16") == pytest.approx(50.7e6, abs=0.05e6)
    assert bench.whole_step_bytes(riser3d, "f32") == pytest.approx(12.92e9, abs=0.005e9)
    # collide_stream alone: populations twice, the offset, rho, u_act, F_p->g,
    # beta and 1 - eps per cell, a velocity per particle
    assert bench.collide_stream_bytes(riser, "f32")[1:] == (104, 8)
    assert bench.collide_stream_bytes(riser3d, "f32")[1:] == (192, 12)
    assert bench.collide_stream_bytes(riser3d, "f16")[1:] == (116, 12)
