"""Serving: continuous batching of independent beds (lbdps_server_*).

A bed's result must be the same when it runs alone, directly through
lbdps_create/lbdps_step, or inside a mix of beds that arrive while it runs;
admission must keep the resident footprint within the HBM budget; a request
that can never fit is rejected; an allocator failure (injected on the host
through the allocator callback) fails that request and leaves the server
serving the others.
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


def _lb():
    from paper_1303_2653_gb300 import lbdps
    return lbdps


def _mix():
    return [W.scaled_riser2d(nx=64, ny=128, seed=11),
            W.bubbling2d(nx=32, ny=64, n_particles=300, seed=12, storage=W.STORE_F32),
            W.scaled_riser2d(nx=96, ny=64, seed=13, storage=W.STORE_F16),
            W.scaled_riser3d(nx=12, ny=12, nz=24, n_particles=500, solid_fraction=0.05, seed=14)]


def _drain(server, want, max_polls=200000):
    done = {}
    for _ in range(max_polls):
        for r in server.poll(wait_s=0.001):
            done[r["id"]] = r
        if want <= set(done):
            return done
    raise AssertionError("server did not finish")


@pytest.mark.parametrize("batching", [True, False])
def test_result_alone_equals_mix_and_direct(batching):
    # batching on: the 2D FP32 / FP16 beds advance in the batched kernels
    # (one launch per kernel class over all of them), the 3D bed on its own
    # stream; off: every bed on its own stream.  A tick of 5 steps (odd) moves
    # the buffer parity at every tick.
    L = _lb()
    beds = _mix()
    target, K = beds[0], 47
    direct = L.Bed(target)
    direct.step(K)
    f_d = direct.populations()
    P_d, v_d = direct.particles()
    direct.close()

    s = L.Server(hbm_budget=4 << 30, max_active=8, steps_per_tick=5, batching=batching)
    rid = s.submit(target, K, keep=True)
    assert _drain(s, {rid})[rid]["status"] == 0
    alone = s.take(rid)
    np.testing.assert_array_equal(alone.populations(), f_d)
    P_a, v_a = alone.particles()
    np.testing.assert_array_equal(P_a, P_d)
    np.testing.assert_array_equal(v_a, v_d)
    alone.close()

    ids = [s.submit(beds[1], 80), s.submit(beds[2], 33)]
    rid = s.submit(target, K, keep=True)
    s.poll(wait_s=0.0)
    ids.append(s.submit(beds[3], 25))          # arrives while the target runs
    done = _drain(s, set(ids) | {rid})
    assert all(done[i]["status"] == 0 for i in ids + [rid])
    mixed = s.take(rid)
    np.testing.assert_array_equal(mixed.populations(), f_d)
    P_m, v_m = mixed.particles()
    np.testing.assert_array_equal(P_m, P_d)
    np.testing.assert_array_equal(v_m, v_d)
    # the handle taken from the server steps on by itself like the direct bed
    mixed.step(3)
    direct = L.Bed(target)
    direct.step(K + 3)
    np.testing.assert_array_equal(mixed.populations(), direct.populations())
    direct.close()
    mixed.close()
    ticks, captures, members = s.batch_info()
    if batching:
        assert ticks > 0 and captures >= 1
    else:
        assert ticks == 0
    s.close()


def test_batched_beds_equal_beds_alone():
    # many small beds of both kinds, three storage formats, LES on and off,
    # particle counts from 0 up, different step counts, all admitted at once
    # into the batch: each equals the same bed stepped alone, bit for bit
    L = _lb()
    beds = [W.scaled_riser2d(nx=48, ny=64, seed=51),
            W.scaled_riser2d(nx=40, ny=96, seed=52, storage=W.STORE_F16, cs_smag=0.1),
            W.scaled_riser2d(nx=64, ny=32, seed=53, storage=W.STORE_BF16),
            W.bubbling2d(nx=32, ny=64, n_particles=400, seed=54, storage=W.STORE_F32, cs_smag=0.1),
            W.bubbling2d(nx=24, ny=40, n_particles=150, seed=55, storage=W.STORE_F16),
            W.channel2d(nx=16, ny=8, h=1.0, dt=1.0, nu=0.05, body_accel=1e-6, storage=W.STORE_F32),
            W.riser2d(nx=100, ny=130, n_particles=3000, seed=56, storage=W.STORE_F32)]
    steps = [37, 64, 20, 45, 9, 30, 33]
    s = L.Server(hbm_budget=8 << 30, max_active=16, steps_per_tick=8)
    ids = [s.submit(w, k, keep=True) for w, k in zip(beds, steps)]
    done = _drain(s, set(ids))
    assert all(done[i]["status"] == 0 for i in ids)
    ticks, captures, members = s.batch_info()
    assert ticks >= 8 and captures == 1
    for w, k, rid in zip(beds, steps, ids):
        got = s.take(rid)
        ref = L.Bed(w)
        ref.step(k)
        np.testing.assert_array_equal(got.populations(), ref.populations(), err_msg=w.name)
        Pg, vg = got.particles()
        Pr, vr = ref.particles()
        np.testing.assert_array_equal(Pg, Pr)
        np.testing.assert_array_equal(vg, vr)
        assert got.stats()["steps"] == k
        got.close()
        ref.close()
    s.close()


def test_batch_membership_rule():
    # a bed above the size limit, or with more particles than cells, keeps its
    # own stream; lowering the limit sends the small bed there too
    L = _lb()
    small = W.scaled_riser2d(nx=48, ny=64, seed=61)
    dense = W.riser2d(nx=32, ny=32, n_particles=1100, seed=62, h=1.322e-4)
    assert dense.n_particles > dense.ncell
    for max_cells, batched in ((0, True), (1000, False)):
        s = L.Server(hbm_budget=4 << 30, max_active=8, steps_per_tick=4, batch_max_cells=max_cells)
        ids = [s.submit(small, 12), s.submit(dense, 12)]
        s.poll(wait_s=0.0)
        _, _, members = s.batch_info()
        assert members == (1 if batched else 0)
        done = _drain(s, set(ids))
        assert all(done[i]["status"] == 0 for i in ids)
        s.close()


def test_admission_stays_within_budget():
    L = _lb()
    w = W.scaled_riser2d(nx=64, ny=64, seed=21)
    need = L.memory_estimate(w)
    s = L.Server(hbm_budget=2 * need + need // 2, max_active=16, steps_per_tick=4)
    ids = [s.submit(w, 30) for _ in range(5)]
    seen_active, done = 0, {}
    for _ in range(200000):
        q, a, used = s.load()
        assert used <= 2 * need + need // 2
        seen_active = max(seen_active, a)
        for r in s.poll(wait_s=0.0005):
            done[r["id"]] = r
        if set(ids) <= set(done):
            break
    assert set(ids) <= set(done)
    assert seen_active == 2
    assert all(done[i]["status"] == 0 and done[i]["steps"] == 30 for i in ids)
    assert s.load() == (0, 0, 0)
    s.close()


def test_request_beyond_budget_is_rejected():
    L = _lb()
    w = W.scaled_riser2d(nx=64, ny=64, seed=22)
    s = L.Server(hbm_budget=L.memory_estimate(w) - 1, max_active=4, steps_per_tick=4)
    with pytest.raises(L.LbdpsError) as ei:
        s.submit(w, 10)
    assert ei.value.code == L.ERR_CAPACITY
    s.close()


def test_allocator_failure_fails_only_that_request():
    L = _lb()
    w = W.scaled_riser2d(nx=64, ny=64, seed=23)
    s = L.Server(hbm_budget=1 << 30, max_active=4, steps_per_tick=4)
    ok1 = s.submit(w, 20)
    bad = s.submit(w, 20, alloc=lambda n: None, free=lambda p: None)   # refuses every allocation
    ok2 = s.submit(w, 20)
    done = _drain(s, {ok1, bad, ok2})
    assert done[ok1]["status"] == 0 and done[ok2]["status"] == 0
    assert done[bad]["status"] == L.ERR_OOM
    s.close()


def test_misaligned_allocator_block_is_rejected_before_any_kernel():
    # A block off a 256-byte boundary would break the 16-byte vector accesses
    # of the kernels: the bed must fail at creation with ERR_INVALID.
    import torch
    L = _lb()
    w = W.scaled_riser2d(nx=64, ny=64, seed=24)
    s = L.Server(hbm_budget=1 << 30, max_active=4, steps_per_tick=4)
    held = {}

    def alloc(n):
        base = torch.cuda.caching_allocator_alloc(int(n) + 256)
        held[base + 16] = base
        return base + 16

    def free(p):
        torch.cuda.caching_allocator_delete(held.pop(p))

    bad = s.submit(w, 10, alloc=alloc, free=free)
    ok = s.submit(w, 10)
    done = _drain(s, {bad, ok})
    assert done[bad]["status"] == L.ERR_INVALID
    assert done[ok]["status"] == 0
    assert not held
    s.close()
