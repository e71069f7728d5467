"""Autotuner (sort cadence K, pass grid): it picks from its candidate set,
reports a positive time per particle-step, and — because the deposit is an
integer sum and random numbers are keyed on particle ids — a tuned run ends
bit-identical to an untuned run advanced the same number of steps."""
import numpy as np
import pytest

from paper_2308_13092_gb300 import inputs as I
from helpers import gpu_from_config, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def test_run_autotune_keeps_physics_bit_identical():
    # room for the discharge's growth over the ~3800 trial steps (every
    # candidate tried twice): a full species drops births in thread order,
    # which no two runs share
    cfg = I.with_headroom(I.config_small(seed=7), 8.0)
    a = gpu_from_config(cfg)
    b = gpu_from_config(cfg)
    t = a.autotune(16)
    assert t["sort_every"] in (8, 16, 32, 64)
    assert t["pass_ctas"] >= 0 and t["ns_per_particle_step"] > 0
    done = a.diagnostics(profiles=False)["step"]
    assert done >= 4 * 3 * 16
    b.step(done)
    a.step(50)
    b.step(50)
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        ia, ib = np.argsort(pa["id"]), np.argsort(pb["id"])
        for k in ("cell", "xi", "vx", "vy", "vz", "id"):
            assert np.array_equal(pa[k][ia], pb[k][ib]), k
    assert a.diagnostics(profiles=False)["species"] == b.diagnostics(profiles=False)["species"]


def test_engine_autotune_picks_a_candidate():
    from paper_2308_13092_gb300 import ecpic
    # the runs outlive the trials (every candidate twice: ~3800 steps)
    cfgs = I.batched_manifest(12, seed=5, steps=6000, scale=0.05)
    eng = ecpic.Engine(max_slots=12, max_cells=1024)
    for c in cfgs:
        eng.submit(c)
    eng.pump(0)
    t = eng.autotune(32)
    assert t["sort_every"] in (8, 16, 32, 64)
    assert t["ns_per_particle_step"] > 0
    r, q = eng.pump(10)
    assert r == 12 and q == 0
    eng.close()


def test_engine_autotune_advances_the_steps_the_bench_plans_for():
    """The bench sizes its manifest so that no run retires inside the
    autotuner's trials, from its own count of the steps they take (two trials
    per cadence and grid, each whole sort and sample cycles): the engine
    advances exactly that many."""
    import bench
    from paper_2308_13092_gb300 import ecpic
    cfgs = I.batched_manifest(4, seed=9, steps=8000, scale=0.02)
    for c in cfgs:
        c.sample_every = 40
    eng = ecpic.Engine(max_slots=4, max_cells=1024)
    tks = [eng.submit(c) for c in cfgs]
    eng.pump(0)
    eng.autotune(64, ks=[10, 20])
    got = eng.poll(tks[0], diagnostics=True)["diag"]["step"]
    assert got == bench.autotune_steps(64, Ks=(10, 20), sample_every=40), got
    eng.close()
