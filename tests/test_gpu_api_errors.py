"""Error behaviour of the C ABI: calls out of order return ECPIC_ERR_STATE,
bad arguments ECPIC_ERR_ARG, and a rejected call leaves the run usable
(every call returns a status; nothing is half-applied)."""
import numpy as np
import pytest

from paper_2308_13092_gb300 import inputs as I
from helpers import gpu_from_config, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _code(fn, *a, **kw):
    from paper_2308_13092_gb300 import ecpic
    with pytest.raises(ecpic.EcpicError) as e:
        fn(*a, **kw)
    return e.value.code


def _small():
    return I.ccp("api", N=32, n0=5e13, dt=1.0 / (400 * I.F_RF), ppc=0, v0=300.0, p_mtorr=60.0,
                 n_steps=10, seed=1, L=0.02, n_per_species=2000)


def test_out_of_order_calls():
    from paper_2308_13092_gb300 import ecpic
    cfg = _small()
    r = gpu_from_config(cfg, init=False)
    assert _code(r.step, 1) == ecpic.ECPIC_ERR_STATE
    assert _code(r.sort_now) == ecpic.ECPIC_ERR_STATE
    assert _code(r.reserve, 0, 10 ** 6) == ecpic.ECPIC_ERR_STATE
    r.init(cfg.seed, cfg.dt, [s.n0 for s in cfg.species], [s.T_eV for s in cfg.species])
    assert _code(r.init, cfg.seed, cfg.dt, [s.n0 for s in cfg.species],
                 [s.T_eV for s in cfg.species]) == ecpic.ECPIC_ERR_STATE
    r.step(5)
    r.sync()
    assert r.diagnostics(profiles=False)["step"] == 5
    r.close()


def test_bad_grids_and_schemes_are_rejected():
    from paper_2308_13092_gb300 import ecpic
    r = ecpic.Run()
    e = I.uniform_edges(32, 0.02)
    assert _code(r.set_grid, e[::-1].copy()) == ecpic.ECPIC_ERR_ARG          # decreasing
    bad = e.copy()
    bad[0] = 1e-6
    assert _code(r.set_grid, bad) == ecpic.ECPIC_ERR_ARG                     # edges[0] != 0
    assert _code(r.set_grid, I.uniform_edges(2049, 0.3)) == ecpic.ECPIC_ERR_ARG  # > max cells
    assert _code(r.set_scheme, 7) == ecpic.ECPIC_ERR_ARG
    r.close()
    # EC2 needs a uniform grid: rejected when the run is initialised
    cfg = _small()
    cfg.edges = I.tanh_edges(32, 0.02, 0.02 / 200)
    cfg.scheme = I.EC2
    r = gpu_from_config(cfg, init=False)
    assert _code(r.init, cfg.seed, cfg.dt, [s.n0 for s in cfg.species],
                 [s.T_eV for s in cfg.species]) == ecpic.ECPIC_ERR_ARG
    r.close()


def test_bad_particles_leave_the_run_usable():
    from paper_2308_13092_gb300 import ecpic
    cfg = _small()
    r = gpu_from_config(cfg)
    p = r.get_particles(0)
    n = p["id"].size
    cell = p["cell"].copy()
    cell[3] = cfg.N                                              # past the last cell
    assert _code(r.set_particles, 0, cell, p["xi"], p["vx"], p["vy"], p["vz"], p["id"]) \
        == ecpic.ECPIC_ERR_ARG
    xi = p["xi"].copy()
    xi[5] = 1.0                                                  # xi must be < 1
    assert _code(r.set_particles, 0, p["cell"], xi, p["vx"], p["vy"], p["vz"], p["id"]) \
        == ecpic.ECPIC_ERR_ARG
    assert _code(r.set_particles, 7, p["cell"], p["xi"], p["vx"], p["vy"], p["vz"], p["id"]) \
        == ecpic.ECPIC_ERR_ARG                                   # unknown species
    assert _code(r.reserve, 5, 10 ** 6) == ecpic.ECPIC_ERR_ARG
    assert _code(r.reserve, 0, 2 ** 31) == ecpic.ECPIC_ERR_ARG    # above 2^31 - 1
    # nothing was applied: same particles, and the run still steps
    q = r.get_particles(0)
    assert q["id"].size == n and np.array_equal(np.sort(q["id"]), np.sort(p["id"]))
    r.step(3)
    r.sync()
    assert r.diagnostics(profiles=False)["step"] == 3
    r.close()


def test_engine_rejects_runs_beyond_its_limits():
    from paper_2308_13092_gb300 import ecpic
    eng = ecpic.Engine(max_slots=2, max_cells=64)
    big = I.ccp("too-many-cells", N=128, n0=5e13, dt=1.0 / (400 * I.F_RF), ppc=0, v0=300.0,
                p_mtorr=60.0, n_steps=10, seed=1, L=0.05, n_per_species=1000)
    assert _code(eng.submit, big) == ecpic.ECPIC_ERR_ARG  # more cells than max_cells
    t_ok = eng.submit(_small())
    for _ in range(20):
        r, q = eng.pump(10)
        if r == 0 and q == 0:
            break
    assert eng.poll(t_ok)["state"] == 2
    eng.close()
