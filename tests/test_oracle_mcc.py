"""Pins for the oracle's null-collision Monte Carlo (Sec. 2a step 6, Sec. 2b):
collision rate against n_g sigma v, exact energy bookkeeping of excitation
and ionisation, the mean elastic energy loss 2m/M, and the gas Maxwellian of
charge exchange."""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I

NG = I.gas_density(30.0)


def _gas_run(kind, sigma_value, E_top, n, E0, dt, heavy=False, thr=0.0, ion_sp=False,
             direction=None, seed=11, table=None):
    """n particles of energy E0 (eV) in an empty gap (zero weight, no field)."""
    o = oracle.OracleRun()
    o.set_grid(I.uniform_edges(8, 1.0), oracle.DIRICHLET)
    m = I.M_ION if heavy else I.ME
    q = I.QE if heavy else -I.QE
    o.add_species(q, m, 0.0, 3 * n)
    if ion_sp:
        o.add_species(I.QE, I.M_ION, 0.0, 3 * n)
    o.set_gas(NG, 300.0, I.M_ION)
    dE = 0.5
    nt = int(round(E_top / dE)) + 1
    sig = table if table is not None else np.full(nt, sigma_value, np.float32)
    o.add_process(0, kind, thr, dE, sig, 1 if kind == oracle.IONIZATION else -1)
    o.init(seed, dt, [0] + ([0] if ion_sp else []), [0.0] + ([0.0] if ion_sp else []))
    rng = np.random.default_rng(seed)
    sp = np.sqrt(2 * E0 * I.QE / m)
    if direction is None:
        d = rng.normal(size=(3, n))
        d /= np.linalg.norm(d, axis=0)
    else:
        d = np.tile(np.asarray(direction, float)[:, None], (1, n))
    X = np.full(n, 0.5)
    o.set_particles(0, X, sp * d[0], sp * d[1], sp * d[2], np.arange(n, dtype=np.uint64))
    return o, sp * d


def test_collision_rate_equals_ng_sigma_v():
    """Constant sigma, monoenergetic at the table top (so nu_max = n_g sigma v):
    collided fraction = 1 - exp(-n_g sigma v dt) within 4 binomial sigmas."""
    n, E0, sigma, dt = 200000, 50.0, 5e-20, 2e-9
    o, v0 = _gas_run(oracle.ELASTIC, sigma, E0, n, E0, dt)
    nu, thr = o.nu_max(0)
    v = np.sqrt(2 * E0 * I.QE / I.ME)
    assert np.isclose(nu, NG * sigma * v, rtol=1e-6)
    o.step(1)
    c = o.counters()["species"][0]
    p = 1 - np.exp(-NG * sigma * v * dt)
    k = c["collisions"][0]
    assert abs(k - n * p) <= 4 * np.sqrt(n * p * (1 - p))
    # every collision changes the direction; nothing else does
    pv = o.get_particles(0)
    changed = np.sum(~np.isclose(pv["vx"], v0[0], rtol=1e-12, atol=0))
    assert changed == k
    # candidates follow the 24-bit integer threshold of P = 1 - exp(-nu_max dt)
    assert thr == int(np.ceil((1 - np.exp(-nu * dt)) * 2 ** 24))


def test_null_collision_fraction_below_table_top():
    """Particles at 1/4 of the top energy collide with probability
    P_null * nu/nu_max = P_null / 2 (constant sigma, v ~ sqrt(E))."""
    n, sigma, dt = 200000, 5e-20, 2e-9
    o, _ = _gas_run(oracle.ELASTIC, sigma, 200.0, n, 50.0, dt)
    nu, thr = o.nu_max(0)
    o.step(1)
    c = o.counters()["species"][0]
    P = thr / 2 ** 24
    p = P * 0.5
    assert abs(c["collisions"][0] - n * p) <= 4 * np.sqrt(n * p * (1 - p))
    assert abs(c["candidates"] - n * P) <= 4 * np.sqrt(n * P * (1 - P))


def test_candidates_follow_philox_stream():
    """The candidate test is (r0 >> 8) < threshold with r = Philox(key = seed,
    counter = (id lo, id hi, step, species << 8))."""
    n, dt, seed = 3000, 2e-9, 99
    o, _ = _gas_run(oracle.ELASTIC, 5e-20, 50.0, n, 50.0, dt, seed=seed)
    _, thr = o.nu_max(0)
    expect = 0
    for i in range(n):
        r = oracle.philox4x32_10((i, 0, 0, 0), (seed & 0xFFFFFFFF, seed >> 32))
        expect += (r[0] >> 8) < thr
    o.step(1)
    assert o.counters()["species"][0]["candidates"] == expect


def test_excitation_removes_threshold_energy():
    n, E0, thr = 50000, 30.0, 20.0
    o, v0 = _gas_run(oracle.EXCITATION, 1e-19, 30.0, n, E0, 5e-9, thr=thr)
    o.step(1)
    p = o.get_particles(0)
    E = 0.5 * I.ME * (p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2) / I.QE
    hit = ~np.isclose(p["vx"], v0[0], rtol=1e-12, atol=0)
    assert hit.sum() == o.counters()["species"][0]["collisions"][0] > 100
    assert np.allclose(E[hit], E0 - thr, rtol=1e-12)
    assert np.allclose(E[~hit], E0, rtol=1e-12)


def test_no_excitation_below_threshold():
    n = 20000
    o, _ = _gas_run(oracle.EXCITATION, 1e-19, 30.0, n, 19.9, 5e-9, thr=20.0)
    o.step(1)
    c = o.counters()["species"][0]
    assert c["collisions"][0] == 0 and c["candidates"] > 0


def test_ionisation_energy_bookkeeping_and_births():
    n, E0, Eiz = 40000, 80.0, 25.0
    o, v0 = _gas_run(oracle.IONIZATION, 1e-19, 80.0, n, E0, 5e-9, thr=Eiz, ion_sp=True)
    o.step(1)
    c = o.counters()["species"]
    k = c[0]["collisions"][0]
    assert k > 100 and c[0]["births"] == k and c[0]["n"] == n + k and c[1]["n"] == k
    e = o.get_particles(0)
    ion = o.get_particles(1)
    ids = e["id"]
    by_id = {int(i): j for j, i in enumerate(ids)}
    E = 0.5 * I.ME * (e["vx"] ** 2 + e["vy"] ** 2 + e["vz"] ** 2) / I.QE
    parents = np.nonzero(~np.isclose(e["vx"][:n], v0[0], rtol=1e-12, atol=0))[0]
    assert parents.size == k
    for j in parents[:500]:
        pid = int(ids[j])
        child = by_id[oracle.child_id(pid, 0, 1)]
        assert np.isclose(E[j] + E[child], E0 - Eiz, rtol=1e-11)
        assert e["X"][child] == e["X"][j]
    ion_ids = set(int(i) for i in ion["id"])
    assert all(oracle.child_id(int(ids[j]), 0, 2) in ion_ids for j in parents)
    # new ions carry the 300 K gas Maxwellian
    sd = np.sqrt(I.KB * 300.0 / I.M_ION)
    for comp in ("vx", "vy", "vz"):
        assert abs(ion[comp].mean()) < 5 * sd / np.sqrt(k)
        assert abs(ion[comp].std() / sd - 1) < 5 / np.sqrt(2 * k)


def test_elastic_mean_energy_loss_is_2m_over_M():
    n, E0 = 200000, 10.0
    o, v0 = _gas_run(oracle.ELASTIC, 5e-19, 10.0, n, E0, 5e-9)
    o.step(1)
    p = o.get_particles(0)
    hit = ~np.isclose(p["vx"], v0[0], rtol=1e-12, atol=0)
    E = 0.5 * I.ME * (p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2) / I.QE
    loss = (E0 - E[hit]) / E0
    ratio = 2 * I.ME / I.M_ION
    # isotropic scattering: 1 - cos(chi) is uniform on [0, 2], mean 1, sd 1/sqrt(3)
    assert abs(loss.mean() / ratio - 1) < 5 / np.sqrt(3 * hit.sum())
    assert loss.min() >= 0 and loss.max() <= 2 * ratio * (1 + 1e-9)


def test_charge_exchange_gives_gas_velocity():
    n = 100000
    o, v0 = _gas_run(oracle.CX, 3e-19, 100.0, n, 100.0, 5e-8, heavy=True,
                     direction=(1.0, 0.0, 0.0))
    o.step(1)
    p = o.get_particles(0)
    hit = ~np.isclose(p["vx"], v0[0], rtol=1e-12, atol=0)
    k = hit.sum()
    assert k == o.counters()["species"][0]["collisions"][0] > 1000
    sd = np.sqrt(I.KB * 300.0 / I.M_ION)
    for comp in ("vx", "vy", "vz"):
        assert abs(p[comp][hit].mean()) < 5 * sd / np.sqrt(k)
        assert abs(p[comp][hit].std() / sd - 1) < 5 / np.sqrt(2 * k)


def test_ion_elastic_equal_mass_halves_mean_velocity():
    """Equal masses, isotropic in the centre-of-mass frame, cold-ish gas: the
    mean post-collision velocity is the centre-of-mass velocity ~ v/2, and the
    relative speed is preserved."""
    n, E0 = 100000, 100.0
    o, v0 = _gas_run(oracle.ION_ELASTIC, 2e-19, 100.0, n, E0, 5e-8, heavy=True,
                     direction=(1.0, 0.0, 0.0))
    V = v0[0, 0]
    o.step(1)
    p = o.get_particles(0)
    hit = ~np.isclose(p["vx"], V, rtol=1e-12, atol=0)
    k = hit.sum()
    assert k > 1000
    sd = np.sqrt(I.KB * 300.0 / I.M_ION)
    mean_vx = p["vx"][hit].mean()
    assert abs(mean_vx - V / 2) < 5 * (V / 2 / np.sqrt(3 * k) + sd / np.sqrt(k))
    # speed of the ion in the CM frame is half the relative speed: |v' - v_cm|
    # ranges over [0, V] when the gas is cold
    sp = np.sqrt(p["vx"][hit] ** 2 + p["vy"][hit] ** 2 + p["vz"][hit] ** 2)
    assert sp.max() <= V * 1.05


def test_clamp_counted_above_table():
    n = 20000
    o, _ = _gas_run(oracle.ELASTIC, 5e-20, 20.0, n, 80.0, 2e-9)
    o.step(1)
    c = o.counters()["species"][0]
    assert c["clamps"] == c["candidates"] > 0
