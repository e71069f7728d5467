"""Measurement entry points of the boundary: phase timing inside the replayed
step graphs, the sort state, the autotuner over given sort cadences.

* with phase timing on, every step advanced reports one pass, one collision
  and one field launch, and every sort four launches; the phase sums are
  positive; the physics is unchanged (same counters as the run without timing);
* the sort state follows the cadence: after the autotuner over {5, 10} the
  chosen cadence is one of them, the sort cycle restarts at 0 and advances by
  one per step;
* timing works on the engine too, and turning it off restores the plain
  graphs with the same results.
"""
import pytest

from paper_2308_13092_gb300 import inputs as I
from helpers import gpu_from_config, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _cfg(seed=31):
    c = I.config_small(seed=seed)
    c.sample_every = 10
    return c


def _key(d):
    return [(s["n"], s["births"], s["candidates"], tuple(s["collisions"])) for s in d["species"]]


def test_phase_timing_counts_and_physics():
    a = gpu_from_config(_cfg())
    b = gpu_from_config(_cfg())
    a.set_sort_every(8)
    b.set_sort_every(8)
    b.set_phase_timing(True)
    a.step(8)
    b.step(8)
    b.sync()
    b.phase_times()  # clear
    b.step(40)
    a.step(40)
    a.sync()
    b.sync()
    ph = b.phase_times()
    assert ph["steps"] == 40 and ph["sorts"] == 5
    assert ph["launches"] == [40, 40, 20, 40]
    for k in ("pass_ms", "field_ms", "sort_ms", "collide_ms"):
        assert ph[k] > 0.0, k
    assert _key(a.diagnostics(profiles=False)) == _key(b.diagnostics(profiles=False))
    # sums read again are cleared
    assert b.phase_times()["steps"] == 0
    b.set_phase_timing(False)
    b.step(8)
    a.step(8)
    a.sync()
    b.sync()
    assert _key(a.diagnostics(profiles=False)) == _key(b.diagnostics(profiles=False))


def test_sort_state_and_autotune_over_given_cadences():
    g = gpu_from_config(_cfg(32))
    t = g.autotune(16, ks=[5, 10])
    assert t["sort_every"] in (5, 10)
    st = g.sort_state()
    assert st["sort_every"] == t["sort_every"] and st["since_sort"] == 0
    g.step(3)
    g.sync()
    assert g.sort_state()["since_sort"] == 3
    g.step(t["sort_every"] - 3)
    assert g.sort_state()["since_sort"] == 0


def test_engine_phase_timing_window_of_whole_cycles():
    from paper_2308_13092_gb300 import ecpic
    cfgs = [I.batched_manifest(4, seed=5, steps=400, scale=0.05)[i] for i in range(4)]
    eng = ecpic.Engine(max_slots=4, max_cells=1024)
    for c in cfgs:
        eng.submit(c)
    eng.pump(0)
    eng.tune(0, 10)
    eng.set_phase_timing(True)
    eng.pump(10)
    assert eng.sort_state()["since_sort"] == 0
    eng.phase_times()
    eng.pump(30)
    ph = eng.phase_times()
    assert ph["steps"] == 30 and ph["sorts"] == 3
    assert ph["launches"][2] == 12
    eng.close()
