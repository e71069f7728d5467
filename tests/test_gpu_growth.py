"""Particle capacity that grows with the discharge (ecpic_reserve,
ecpic_set_auto_grow, the engine's automatic growth).

The small discharge builds up by ionisation, so a species sized at its
initial load plus 500 fills within a few hundred steps: without growth the
run stops with ECPIC_ERR_CAPACITY.  Growing the capacity copies the run's
state into a larger block; the trajectory does not depend on the capacity, so
the grown run must equal, counter for counter and particle for particle, the
same run given ample capacity from the start."""
import numpy as np
import pytest

from paper_2308_13092_gb300 import inputs as I
from helpers import gpu_from_config, require_gpu

pytestmark = pytest.mark.gpu

STEPS = 1000


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _cfg(extra):
    c = I.config_small(seed=8)
    c.sample_every = 10
    c.n_steps = STEPS
    for sp in c.species:
        sp.capacity = sp.n0 + extra
    return c


def _key(d):
    return [(s["n"], s["absorbed_left"], s["absorbed_right"], s["births"], s["candidates"],
             tuple(s["collisions"])) for s in d["species"]]


def _same_particles(a, b):
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        ia, ib = np.argsort(pa["id"]), np.argsort(pb["id"])
        for k in ("cell", "xi", "vx", "vy", "vz", "id"):
            assert np.array_equal(pa[k][ia], pb[k][ib]), (s, k)


@pytest.fixture(scope="module")
def ample():
    require_gpu()
    g = gpu_from_config(_cfg(40_000))
    g.step(STEPS)
    g.sync()
    d = g.diagnostics()
    assert d["species"][0]["n"] > _cfg(500).species[0].capacity  # the tight run must grow
    return g, d


def test_tight_capacity_fails_without_growth():
    from paper_2308_13092_gb300 import ecpic
    g = gpu_from_config(_cfg(500))
    g.step(STEPS)
    assert g.sync(allow=(ecpic.ECPIC_ERR_CAPACITY,)) == ecpic.ECPIC_ERR_CAPACITY
    g.close()


def test_reserve_between_steps_keeps_the_trajectory(ample):
    big, d_big = ample
    g = gpu_from_config(_cfg(500))
    g.step(100)
    g.reserve(0, 40_000 + g.get_particles(0)["id"].size)
    g.reserve(1, 40_000 + g.get_particles(1)["id"].size)
    g.step(STEPS - 100)
    g.sync()
    d = g.diagnostics()
    assert _key(d) == _key(d_big)
    np.testing.assert_array_equal(d["density"], d_big["density"])
    _same_particles(g, big)
    g.close()


def test_auto_grow_single_run(ample):
    big, d_big = ample
    g = gpu_from_config(_cfg(500))
    g.set_auto_grow(True)
    g.step(STEPS)
    g.sync()
    d = g.diagnostics()
    assert _key(d) == _key(d_big)
    np.testing.assert_array_equal(d["density"], d_big["density"])
    _same_particles(g, big)
    g.close()


def test_engine_grows_its_runs(ample):
    from paper_2308_13092_gb300 import ecpic
    _, d_big = ample
    eng = ecpic.Engine(max_slots=2, max_cells=256)
    tk = eng.submit(_cfg(500))
    eng.pump(0)
    b0 = eng.stats()["bytes_resident"]
    for _ in range(100):
        r, q = eng.pump(250)
        if r == 0 and q == 0:
            break
    res = eng.poll(tk, diagnostics=True, profiles=True)
    eng.close()
    assert res["state"] == 2, res["state"]
    d = res["diag"]
    assert _key(d) == _key(d_big)
    np.testing.assert_allclose(d["density"], d_big["density"], rtol=1e-12,
                               atol=1e-12 * np.abs(d_big["density"]).max())
    assert b0 > 0
