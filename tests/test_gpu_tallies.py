"""Diagnostic tallies on the GPU against the oracle, one step from an
identical state (Sec. 3a diagnostics):

* EEDF of the central cells and the power density J.E per cell, on a sample
  step of a colliding discharge, for the linear schemes and for EC2 / MC2
  (whose pass samples in its own instance): EEDF counts equal up to a few
  bin-edge or face flips (FP32 vs FP64 energies and positions), J.E within
  FP32 rounding of the field scale;
* ion impact energy and angle at x = 0 for ions leaving through the RF
  electrode with spread energies and angles: same bins up to edge flips, and
  one count per absorbed ion."""
import numpy as np
import pytest

from paper_2308_13092_gb300 import inputs as I
from helpers import oracle_from_config, gpu_from_config, require_gpu
from test_gpu_parity import _small, _set_same_state

pytestmark = pytest.mark.gpu

TALLY = dict(eedf_center=-1.0, eedf_halfwidth=0.0125, eedf_dE=1.0, eedf_bins=60, iedf_dE=1.0,
             iedf_bins=100, iad_bins=90)


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("scheme,grid", [(I.EC, "uniform"), (I.MC, "uniform"), (I.EC2, "uniform"),
                                         (I.MC2, "uniform"), (I.EC, "tanh"), (I.MC, "tanh")])
def test_eedf_and_power_one_step(scheme, grid):
    edges = I.tanh_edges(70, 0.05, 0.05 / 400) if grid == "tanh" else None
    cfg = _small(scheme=scheme, n=20000, edges=edges)
    cfg.sample_every = 1
    cfg.tallies = TALLY
    g, o = gpu_from_config(cfg), oracle_from_config(cfg)
    _set_same_state(cfg, g, o, seed=21)
    g.step(1)
    o.step(1)
    d = g.diagnostics()
    t = o.tallies()
    assert d["n_samples"] == t["n_samples"] == 1
    assert d["eedf_cells"] == t["eedf_cells"]
    ge, oe = d["eedf"][0], t["eedf"][0]
    assert oe.sum() > 1000
    assert abs(ge.sum() - oe.sum()) <= 2
    assert np.abs(ge - oe).sum() <= 4 + 2e-3 * oe.sum(), (ge, oe)
    assert d["eedf"][1].sum() == 0
    for s in range(2):
        gp, op = d["power"][s], t["power"][s]
        scale = np.abs(op).max()
        assert scale > 0
        np.testing.assert_allclose(gp, op, rtol=0, atol=2e-4 * scale)


@pytest.mark.parametrize("scheme", [I.EC, I.MC, I.EC2, I.MC2])
def test_ion_impacts_one_step(scheme):
    cfg = _small(scheme=scheme, collisions=False, n=8)
    cfg.sample_every = 1
    cfg.tallies = TALLY
    g, o = gpu_from_config(cfg), oracle_from_config(cfg)
    rng = np.random.default_rng(4)
    n = 3000
    E = rng.uniform(0.5, 95.0, n)
    th = np.deg2rad(rng.uniform(0.0, 89.0, n))
    ph = rng.uniform(0, 2 * np.pi, n)
    v = np.sqrt(2 * E * I.QE / I.M_ION)
    vx = (-v * np.cos(th)).astype(np.float32)
    vy = (v * np.sin(th) * np.cos(ph)).astype(np.float32)
    vz = (v * np.sin(th) * np.sin(ph)).astype(np.float32)
    cell = np.zeros(n, np.int32)
    xi = np.full(n, 1e-6, np.float32)
    ids = np.arange(n, dtype=np.uint64) + 5000
    for s in range(2):
        if s == 1:
            g.set_particles(s, cell, xi, vx, vy, vz, ids)
            o.set_particles_cell(s, cell, xi, vx, vy, vz, ids)
        else:
            z = np.zeros(0)
            g.set_particles(s, z.astype(np.int32), z.astype(np.float32), z.astype(np.float32),
                            z.astype(np.float32), z.astype(np.float32), z.astype(np.uint64))
            o.set_particles_cell(s, z.astype(np.int32), z, z, z, z, z.astype(np.uint64))
    g.step(1)
    o.step(1)
    d = g.diagnostics()
    t = o.tallies()
    gs, os_ = d["species"][1], o.counters()["species"][1]
    assert gs["absorbed_left"] == os_["absorbed_left"] == n
    assert gs["impacts_dropped"] == 0
    for k in ("iedf", "iad"):
        gh, oh = d[k][1], t[k][1]
        assert gh.sum() == oh.sum() == n, k
        assert np.abs(gh - oh).sum() <= 6, (k, np.nonzero(gh != oh))
    assert d["iedf"][0].sum() == 0 and d["iad"][0].sum() == 0
