"""Long runs: bed statistics of the GPU path against the FP64 oracle.

After many steps the particle trajectories of the time-driven hard spheres
(§2.2, Eq. 17-18) part ways between any two arithmetics, FP64 against FP64
with a different rounding order included, so pointwise comparison ends after
a few steps.  What must agree is the state of the bed as a whole: the
lattice mean of the gas voidage eps_g (Eq. 10-11 of the current positions)
and the particle-weighted mean slip |u_act - v| (Eq. 26), within 1 %.

The riser section here is the 64 x 512 cut of the periodic riser (12,500
particles, the same solid fraction, cell size and gas as the full
256 x 2048 bed), stepped 1,000 times by the oracle and by the GPU in FP32,
FP16 and BF16 storage of the population deviations.  Both the values after
the last step and their averages over the second half of the run are
compared.  The served form is checked the same way: beds stored in FP16 and
advanced by the serving loop beside other beds against the same beds run
alone in plain FP32.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_2653_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 1000
EVERY = 10        # statistics sampled every EVERY steps on both sides
REL = 0.01        # bed statistics within 1 %


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


def _riser():
    return W.scaled_riser2d(nx=64, ny=512, seed=1303002)


@pytest.fixture(scope="module")
def oracle_series():
    """(mean_eps_g, mean_slip) of the FP64 oracle after every EVERY steps."""
    ob = O.OracleBed(_riser())
    eps, slip = [], []
    for _ in range(STEPS // EVERY):
        ob.step(EVERY)
        s = ob.stats()
        eps.append(s["mean_eps_g"])
        slip.append(s["mean_slip"])
    return np.array(eps), np.array(slip)


def _second_half_mean(x):
    return float(np.mean(x[len(x) // 2:]))


@pytest.mark.parametrize("storage", [W.STORE_F32, W.STORE_F16, W.STORE_BF16])
def test_long_run_bed_statistics_hard_spheres(storage, oracle_series):
    L = _lb()
    # node diagnostics on: the mean slip needs u_act and v_s of every node
    bed = L.Bed(_riser(), storage=storage, diagnostics=True)
    recs = bed.step_monitored(STEPS)
    assert all(r["health"] & 3 == 0 for r in recs)
    eps = np.array([r["mean_eps_g"] for r in recs])[EVERY - 1::EVERY]
    slip = np.array([r["mean_slip"] for r in recs])[EVERY - 1::EVERY]
    eps_o, slip_o = oracle_series
    assert eps.shape == eps_o.shape
    bed.close()
    report = {
        "eps_final": abs(eps[-1] - eps_o[-1]) / eps_o[-1],
        "slip_final": abs(slip[-1] - slip_o[-1]) / slip_o[-1],
        "eps_mean": abs(_second_half_mean(eps) - _second_half_mean(eps_o)) / _second_half_mean(eps_o),
        "slip_mean": abs(_second_half_mean(slip) - _second_half_mean(slip_o)) / _second_half_mean(slip_o),
    }
    print(f"storage {storage}: relative errors after {STEPS} steps {report}; "
          f"oracle mean slip ranged over {np.ptp(slip_o) / slip_o.mean():.2e} of its mean")
    for k, v in report.items():
        assert v <= REL, (k, v, report)


def test_served_fp16_beds_match_fp32_alone():
    # beds of the serving mix (riser and bubbling, LES on as in every served
    # bed) stored in FP16 and advanced by the serving loop together, against
    # the same beds alone in plain FP32
    L = _lb()
    K = 600
    beds = [W.riser2d(nx=96, ny=192, n_particles=2500, seed=1303201, storage=W.STORE_F16,
                      h=1.322e-4, cs_smag=0.1),
            W.riser2d(nx=64, ny=256, n_particles=6000, seed=1303202, storage=W.STORE_F16,
                      h=1.322e-4, cs_smag=0.1),
            W.bubbling2d(nx=64, ny=128, n_particles=1500, seed=1303203, storage=W.STORE_F16,
                         cs_smag=0.1)]
    s = L.Server(hbm_budget=4 << 30, max_active=8, steps_per_tick=32)
    ids = {s.submit(w, K, diagnostics=True): k for k, w in enumerate(beds)}
    # a plain FP32 bed arrives while they run (continuous batching)
    ids[s.submit(W.scaled_riser2d(nx=64, ny=128, seed=1303204), K // 2)] = -1
    done = {}
    for _ in range(400000):
        for r in s.poll(wait_s=0.001):
            done[r["id"]] = r
        if set(ids) <= set(done):
            break
    s.close()
    assert set(ids) <= set(done)
    for rid, k in ids.items():
        assert done[rid]["status"] == 0, done[rid]
        if k < 0:
            continue
        ref = L.Bed(beds[k], storage=W.STORE_F32, diagnostics=True)
        ref.step(K)
        st = ref.stats()
        ref.close()
        e_eps = abs(done[rid]["mean_eps_g"] - st["mean_eps_g"]) / st["mean_eps_g"]
        e_slip = abs(done[rid]["mean_slip"] - st["mean_slip"]) / st["mean_slip"]
        print(f"served FP16 bed {k}: mean voidage {e_eps:.2e}, mean slip {e_slip:.2e}")
        assert e_eps <= REL
        assert e_slip <= REL
