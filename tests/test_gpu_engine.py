"""Batched / served engine through the C ABI (ecpic_engine_*).

Each run's trajectory depends only on its own state: random numbers are keyed
on (particle id, step) and the deposit is an integer sum, so a run gives the
same counters (absorptions, births, collisions per process, candidates) and
particle counts alone, through the single-run API, and in a mix of uneven
runs.  Its averaged density (from the integer deposit) and potential (FP64
field solve of that deposit) agree to FP64 rounding; the temperature is built
from FP32 velocity moments summed with atomics in thread order, so it agrees
to FP32 rounding."""
import numpy as np
import pytest

from paper_2308_13092_gb300 import inputs as I
from helpers import gpu_from_config, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _manifest(n=8, steps=300, scale=0.02, seed=3):
    runs = I.batched_manifest(n, seed=seed, steps=steps, scale=scale)
    for i, c in enumerate(runs):
        c.sample_every = 10
        c.n_steps = steps - 40 * (i % 3)  # uneven lengths
    return runs


def _run_engine(cfgs, **kw):
    from paper_2308_13092_gb300 import ecpic
    eng = ecpic.Engine(max_slots=kw.pop("max_slots", 16), max_cells=1024, **kw)
    tickets = [eng.submit(c) for c in cfgs]
    for _ in range(200):
        r, q = eng.pump(64)
        if r == 0 and q == 0:
            break
    out = [eng.poll(t, diagnostics=True, profiles=True) for t in tickets]
    st = eng.stats()
    eng.close()
    return out, st


def _key(d):
    return [(s["n"], s["absorbed_left"], s["absorbed_right"], s["births"], s["candidates"],
             tuple(s["collisions"])) for s in d["species"]]


def test_run_alone_equals_run_in_mix():
    cfgs = _manifest()
    mix, st = _run_engine(cfgs)
    assert all(o["state"] == 2 for o in mix)
    assert st["runs_finished"] == len(cfgs)
    for i in (0, 3, 7):
        alone, _ = _run_engine([cfgs[i]], max_slots=1)
        a, m = alone[0]["diag"], mix[i]["diag"]
        assert a["step"] == m["step"] == cfgs[i].n_steps
        assert _key(a) == _key(m)
        assert alone[0]["particle_steps"] == mix[i]["particle_steps"]
        for k, tol in (("density", 1e-12), ("phi", 1e-9), ("Tx", 2e-5)):
            np.testing.assert_allclose(a[k], m[k], rtol=tol, atol=tol * np.abs(m[k]).max())


def test_engine_equals_single_run_api():
    cfg = _manifest(n=2)[1]
    eng, _ = _run_engine([cfg])
    g = gpu_from_config(cfg)
    g.step(cfg.n_steps)
    d = g.diagnostics()
    e = eng[0]["diag"]
    assert _key(d) == _key(e)
    np.testing.assert_allclose(d["density"], e["density"], rtol=1e-9,
                               atol=1e-12 * np.abs(e["density"]).max())


def test_memory_budget_admission():
    from paper_2308_13092_gb300 import ecpic
    cfgs = _manifest(n=6, steps=120)
    eng = ecpic.Engine(max_slots=6, max_cells=1024, mem_budget=1)
    with pytest.raises(ecpic.EcpicError):
        eng.submit(cfgs[0])   # larger than the whole budget
    eng.close()
    # budget for about two of the largest runs at a time: all still finish
    big = max(cfgs, key=lambda c: c.n_particles)
    probe = ecpic.Engine(max_slots=1, max_cells=1024)
    probe.submit(big)
    probe.pump(0)
    budget = int(1.5 * probe.stats()["bytes_resident"])
    probe.close()
    eng = ecpic.Engine(max_slots=6, max_cells=1024, mem_budget=budget)
    cfgs = [big] * 4 + cfgs   # four copies of the largest cannot be resident together
    tickets = [eng.submit(c) for c in cfgs]
    seen_queue = False
    for _ in range(300):
        r, q = eng.pump(40)
        seen_queue = seen_queue or q > 0
        if r == 0 and q == 0:
            break
    assert all(eng.poll(t)["state"] == 2 for t in tickets)
    assert seen_queue
    eng.close()


def test_failing_run_is_isolated():
    from paper_2308_13092_gb300 import ecpic
    cfgs = _manifest(n=3, steps=150)
    bad = cfgs[1]
    for sp in bad.species:
        sp.capacity = sp.n0 + 2
    bad.species[0].T_eV = 60.0   # hot electrons ionise from the first step
    bad.n_gas *= 50
    out, _ = _run_engine(cfgs)
    assert out[1]["state"] == ecpic.ECPIC_ERR_CAPACITY
    assert out[0]["state"] == 2 and out[2]["state"] == 2
    good, _ = _run_engine([cfgs[2]], max_slots=1)
    assert _key(good[0]["diag"]) == _key(out[2]["diag"])


def test_runs_admitted_while_others_run_equal_alone():
    """Continuous batching: ten runs arrive in three waves while earlier ones
    are resident and stepping (four slots, so later runs also wait in the
    queue for a slot to free); each finished run equals the same run alone."""
    from paper_2308_13092_gb300 import ecpic
    cfgs = _manifest(n=10, steps=240, seed=11)
    eng = ecpic.Engine(max_slots=4, max_cells=1024)
    tickets = [eng.submit(c) for c in cfgs[:3]]
    eng.pump(50)
    tickets += [eng.submit(c) for c in cfgs[3:7]]
    r, q = eng.pump(50)
    assert r == 4 and q > 0  # full slots, a queue behind them
    tickets += [eng.submit(c) for c in cfgs[7:]]
    for _ in range(200):
        r, q = eng.pump(40)
        if r == 0 and q == 0:
            break
    res = [eng.poll(t, diagnostics=True, profiles=True) for t in tickets]
    eng.close()
    assert all(o["state"] == 2 for o in res)
    for i in (0, 4, 8, 9):
        alone, _ = _run_engine([cfgs[i]], max_slots=1)
        a, m = alone[0]["diag"], res[i]["diag"]
        assert a["step"] == m["step"] == cfgs[i].n_steps
        assert _key(a) == _key(m), i
        for k, tol in (("density", 1e-12), ("phi", 1e-9), ("Tx", 2e-5)):
            np.testing.assert_allclose(a[k], m[k], rtol=tol, atol=tol * np.abs(m[k]).max())
