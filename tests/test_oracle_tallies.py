"""Pins for the oracle's diagnostic tallies (Sec. 3a: EEDF at the discharge
centre, ion impact energy and angle at the RF electrode, power deposition):

* EEDF of a loaded Maxwellian (quiet neutral start, no field) against the
  exact Maxwell-Boltzmann bin probabilities (energy/T is chi-square with 3
  degrees of freedom / 2), and its total against the electrons counted in the
  region's cells from their positions;
* a monoenergetic ion beam at a known angle lands in the expected energy and
  angle bins, one count per absorbed ion, electrons and the far wall not
  counted;
* J.E summed over cells times dt equals the change of the x kinetic energy
  over the push (work-energy theorem of the leapfrog, exact to rounding),
  for EC and MC."""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I
from helpers import oracle_from_config


def _maxwellian_box():
    cfg = I.periodic_plasma(N=64, dx_lambda=1.0, ppc=4000, dt_wpe=0.1, seed=11, ions=True,
                            Te=2.0, Ti=2.0, quiet=True)
    cfg.sample_every = 1
    return cfg


def test_eedf_of_a_maxwellian():
    scipy_special = pytest.importorskip("scipy.special")
    cfg = _maxwellian_box()
    L = cfg.edges[-1]
    o = oracle_from_config(cfg, init=False)
    hw = 4 * (L / 64)  # a few cells around the centre
    o.set_tallies(eedf_center=-1.0, eedf_halfwidth=hw, eedf_dE=0.25, eedf_bins=60)
    o.init(cfg.seed, cfg.dt, [s.n0 for s in cfg.species], [s.T_eV for s in cfg.species])
    o.step(1)
    t = o.tallies()
    c0, c1 = t["eedf_cells"]
    assert c1 >= c0 >= 0
    # the region: cells whose centres are within L/2 +- hw
    centres = 0.5 * (cfg.edges[:-1] + cfg.edges[1:])
    sel = np.nonzero(np.abs(centres - L / 2) <= hw)[0]
    assert (c0, c1) == (sel[0], sel[-1])
    p = o.get_particles(0)
    cell = np.searchsorted(cfg.edges, p["X"], side="right") - 1
    inside = (cell >= c0) & (cell <= c1)
    h = t["eedf"][0]
    assert h.sum() == inside.sum()
    assert t["eedf"][1].sum() == 0  # ions (q > 0) have no EEDF
    # Maxwell-Boltzmann: 2E/T ~ chi-square(3); bins of 0.25 eV at T = 2 eV
    edges = np.arange(61) * 0.25
    cdf = scipy_special.gammainc(1.5, edges / 2.0)
    prob = np.diff(cdf)
    prob[-1] = 1.0 - cdf[-2]
    n = h.sum()
    keep = prob * n >= 20
    chi2 = np.sum((h[keep] - n * prob[keep]) ** 2 / (n * prob[keep]))
    dof = keep.sum() - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof), (chi2, dof)


def test_ion_impacts_energy_and_angle():
    e = I.uniform_edges(32, 0.02)
    o = oracle.OracleRun()
    o.set_grid(e, oracle.DIRICHLET)
    o.add_species(-I.QE, I.ME, 1e6, 64)
    o.add_species(I.QE, I.M_ION, 1e6, 64)
    o.set_tallies(iedf_dE=2.0, iedf_bins=50, iad_bins=90)
    o.init(0, 1e-10, [0, 0], [0.0, 0.0])
    E0, th = 37.3, np.deg2rad(30.5)
    v = np.sqrt(2 * E0 * I.QE / I.M_ION)
    n = 10
    X = np.full(n, 1e-9)
    vx = np.full(n, -v * np.cos(th))
    vy = np.full(n, v * np.sin(th))
    z = np.zeros(n)
    ids = np.arange(n, dtype=np.uint64)
    o.set_particles(1, X, vx, vy, z, ids)
    # ions leaving through x = L and electrons through x = 0 are not counted
    o.set_particles(0, X, vx * 1e3, z, z, ids)
    o.step(1)
    c = o.counters()["species"]
    assert c[1]["absorbed_left"] == n and c[0]["absorbed_left"] == n
    t = o.tallies()
    assert t["iedf"][1].sum() == n and t["iad"][1].sum() == n
    assert t["iedf"][1][int(E0 // 2.0)] == n
    assert t["iad"][1][30] == n
    assert t["iedf"][0].sum() == 0 and t["iad"][0].sum() == 0


@pytest.mark.parametrize("scheme", [I.EC, I.MC])
def test_power_tally_is_the_work_on_the_particles(scheme):
    cfg = I.periodic_plasma(N=48, dx_lambda=2.0, ppc=64, dt_wpe=0.2, seed=5, scheme=scheme,
                            ions=True)
    cfg.sample_every = 1
    o = oracle_from_config(cfg)
    o.step(7)
    o.reset_averages(1)
    before = [o.get_particles(s) for s in range(2)]
    o.step(1)
    after = [o.get_particles(s) for s in range(2)]
    t = o.tallies()
    assert t["n_samples"] == 1
    dx = np.diff(cfg.edges)
    work = cfg.dt * float(np.sum(t["power"] * dx[None, :]))
    dke = 0.0
    for s, sp in enumerate(cfg.species):
        ia, ib = np.argsort(before[s]["id"]), np.argsort(after[s]["id"])
        va, vb = before[s]["vx"][ia], after[s]["vx"][ib]
        dke += 0.5 * sp.m * sp.w * float(np.sum(vb * vb - va * va))
    scale = sum(0.5 * sp.m * sp.w * float(np.sum(before[s]["vx"] ** 2))
                for s, sp in enumerate(cfg.species))
    assert abs(work - dke) <= 1e-9 * scale + 1e-12 * abs(dke), (work, dke, scale)
    assert abs(dke) > 1e-7 * scale  # the field did work
